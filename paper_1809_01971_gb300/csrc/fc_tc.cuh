// FP64-accurate contractions on the BF16 tensor cores (tcgen05, TMEM accumulators).
//
// C = alpha * op(A) op(B) + beta * C with FP64 operands produced by the same loaders as the
// FP64 GEMM.  Each CTA owns a 128 x BN output tile and a K range of at most kTcKC = 448.
// Within it every row i of op(A) (column j of op(B)) is scaled by a power of two 2^-E_i
// (2^-F_j) into (-1/2, 1/2) and written as a fixed-point number with S = 8 balanced digits
// of 7 bits,
//     a = 2^E_i sign(a) (sum_{s<S} d_s 2^(-7-7s) + r),   d_s integer in [-64, 64],
// 0 <= r < 2^-56 (offset-binary digits of F = |a| 2^(63-E_i) + 64 sum_s 2^(56-7s)).
// Digits are integers of at most 7 bits, exact in BF16, so every digit product
// (|.| <= 2^12) is exact on the tensor core, and a sum of at most 8 pairs x 448 terms stays
// below 2^24: the FP32 accumulators in TMEM hold it without rounding.  Products of equal
// weight s + t = L share accumulator L (L < S; pairs with s + t >= S carry weight below 2^-70
// and are dropped), so a tile needs S accumulators of BN columns (36 digit-pair MMAs per K
// step).  The epilogue converts the level sums to integers, combines them exactly in 128-bit
// integer arithmetic, rounds once to FP64, applies 2^(E_i + F_j) and adds the tile to C
// (FP64 atomics under split-K).  The error of a product term is below 2^-55 of
// 2^(E_i + F_j) <= 4 max|A_i,:| max|B_:,j|: the rounding level of an FP64 GEMM, at the
// tensor-core rate instead of the FP64 pipe's 2 FMA per SM per clock.
//
// Operand staging: the digit planes are produced by the CTA's threads (loader -> digits ->
// shared memory in the canonical no-swizzle K-major layout: 8 x 16-byte core matrices,
// LBO = 128 B between K-adjacent, SBO = 512 B between M/N-adjacent core matrices); the
// operands are fused expressions (Khatri-Rao rows, scaled columns), so there is no
// materialised tile for TMA to fetch.  Two stages of kTcKS = 32 along K are double-buffered:
// a dedicated warp issues the MMAs of a stage and commits them to that stage's mbarrier
// while the 512 producer threads form the next stage.  Every wait is bounded; on expiry the kernel
// records an error flag, frees its TMEM and returns.
#pragma once
// Included from fc_common.cuh after the loaders and the split-K pre-scale kernel.
#include "fc_common.cuh"
#include <float.h>

namespace fc {

constexpr int kTcDigits = 8;       // S
constexpr int kTcBM = 128;         // MMA M (TMEM lane = output row)
constexpr int kTcKS = 32;          // K per pipeline stage (two K = 16 MMA steps)
constexpr int kTcKC = 448;         // K per CTA: 8 pairs * 448 * 64^2 < 2^24 (exact FP32 sums)
constexpr int kTcThreads = 512;     // digit producers (4 per row of the 128-row A tile)
constexpr int kTcBlock = kTcThreads + 32;   // + one warp that issues the MMAs
constexpr int kTcBadExp = 0x40000000;   // scale marker of a row / column holding Inf or NaN

// Error flag of the tensor-core GEMMs of this translation unit (bounded wait expired), used
// when a launch names no flag of its own (a handle passes the flag slot of its workspace).
static __device__ int g_tc_error;
// Iteration limit of every bounded mbarrier wait (~1 s of polling).
constexpr int kTcWaitFull = 1 << 24;
// Host side (api.cu): the error flag and the producer-side wait limit that the tensor-core
// launches of the calling thread use.  A handle's calls set the flag to a slot of its own
// workspace for their duration; the limit is kTcWaitFull unless a test lowered it.
int* tc_error_target();
int tc_producer_wait_limit();

FC_DEV uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle.
FC_DEV uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

FC_DEV void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}

FC_DEV void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

// Bounded wait for the phase with the given parity of an mbarrier: at most `limit` polls
// (kTcWaitFull: ~1 s).  Returns false if the phase did not complete within them.
FC_DEV bool tc_wait(uint32_t bar, uint32_t parity, int limit = kTcWaitFull) {
    for (int it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

FC_DEV void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3); v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// Exponent bounds from FP64 bit fields (integer operations only): a value with biased
// exponent field e satisfies |x| < 2^(e - 1022); a product of values with fields ea, eb
// has the bound field ea + eb - 1022.  Non-finite values give kTcBadField.
constexpr int kTcBadField = 1 << 20;
FC_DEV int tc_efield(double x) {
    const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
    return (e == 0x7FF) ? kTcBadField : e;
}
FC_DEV int tc_efield2(double a, double b) {
    const int ea = tc_efield(a), eb = tc_efield(b);
    return (ea == kTcBadField || eb == kTcBadField) ? kTcBadField : ea + eb - 1022;
}
// bound field of one operand element; loaders that form products bound them factorwise
template <class L>
FC_DEV int tc_ebound(const L& ld, int i, int k, int b) { return tc_efield(ld(i, k, b)); }
FC_DEV int tc_ebound(const LdCoreW& ld, int ab, int k, int) {
    const int r0 = *ld.r0p, bb = ab / r0, a = ab - bb * r0;
    return tc_efield2(ld.C0[a + (long long)k * ld.ldc], ld.C1w[bb + (long long)k * ld.ldc]);
}
FC_DEV int tc_ebound(const LdKR& ld, int i, int kj, int b) {
    const int k = kj / ld.S, j = kj - k * ld.S;
    return tc_efield2(ld.E[b * ld.bsE + i + (long long)k * ld.lde], ld.Y[b * ld.bsY + i + (long long)j * ld.ldy]);
}
// Largest bound field of op(X)[i, k] over k in [ka, kb) (rows of op(A) / columns of op(B)
// are both addressed as (i, k) through a transposing adaptor below).
template <class L>
FC_DEV int tc_emax_row(const L& ld, int i, int ka, int kb, int b) {
    int fm = -(1 << 30);
    int k = ka;
    for (; k + 8 <= kb; k += 8) {
        int f[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) f[q] = tc_ebound(ld, i, k + q, b);
#pragma unroll
        for (int q = 0; q < 8; ++q) fm = max(fm, f[q]);
    }
    for (; k < kb; ++k) fm = max(fm, tc_ebound(ld, i, k, b));
    return fm;
}
FC_DEV int tc_emax_row(const LdCoreW& ld, int ab, int ka, int kb, int) {
    const int r0 = *ld.r0p, bb = ab / r0, a = ab - bb * r0;
    const double* p0 = ld.C0 + a;
    const double* p1 = ld.C1w + bb;
    int fm = -(1 << 30);
    int k = ka;
    for (; k + 8 <= kb; k += 8) {
        int f[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            f[q] = tc_efield2(p0[(long long)(k + q) * ld.ldc], p1[(long long)(k + q) * ld.ldc]);
#pragma unroll
        for (int q = 0; q < 8; ++q) fm = max(fm, f[q]);
    }
    for (; k < kb; ++k) fm = max(fm, tc_efield2(p0[(long long)k * ld.ldc], p1[(long long)k * ld.ldc]));
    return fm;
}
// op(B) (K x N, element (k, j)) seen as rows j with inner index k
template <class L>
struct TcTrans {
    L ld;
    FC_DEV double operator()(int j, int k, int b) const { return ld(k, j, b); }
};
template <class L>
FC_DEV int tc_ebound(const TcTrans<L>& t, int j, int k, int b) { return tc_ebound(t.ld, k, j, b); }

// Scale exponent E of a row / column from its largest bound field: every |x| < 2^(E-1).
FC_DEV int tc_scale_exp(int fmax_) {
    return (fmax_ >= kTcBadField) ? kTcBadExp : fmax_ - 1021;
}

// Fixed-point magnitude F = |x| 2^(63-E) < 2^62 (integer operations on the FP64 bit
// pattern) and the sign of x.
FC_DEV unsigned long long tc_fixed(double x, int E, uint32_t& sgn) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    const int sh = (e ? e : 1) - 1012 - E;           // F = m 2^sh
    sgn = (uint32_t)(bits >> 32) & 0x80000000u;
    if (sh >= 0) return m << (sh < 10 ? sh : 10);
    return (sh > -64) ? (m >> (-sh)) : 0ull;
}

// Fixed-point magnitude of a product a b: the top 64 bits of the 106-bit mantissa product
// (exact to 2^-63 of 2^E), shifted by the exponents.
FC_DEV unsigned long long tc_fixed2(double a, double b, int E, uint32_t& sgn) {
    const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)((ba >> 52) & 0x7FF), eb = (int)((bb >> 52) & 0x7FF);
    const unsigned long long ma = (ba & 0xFFFFFFFFFFFFFull) | (ea ? (1ull << 52) : 0ull);
    const unsigned long long mb = (bb & 0xFFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull);
    sgn = (uint32_t)((ba ^ bb) >> 32) & 0x80000000u;
    const unsigned long long P = __umul64hi(ma << 11, mb << 11);      // floor(ma mb / 2^42)
    const int sh = (ea ? ea : 1) + (eb ? eb : 1) - 2045 - E;          // F = P 2^sh
    if (sh >= 0) return P << (sh < 63 ? sh : 63);
    return (sh > -64) ? (P >> (-sh)) : 0ull;
}
template <class L>
FC_DEV unsigned long long tc_fixed_of(const L& ld, int i, int k, int b, int E, uint32_t& sgn) {
    return tc_fixed(ld(i, k, b), E, sgn);
}
FC_DEV unsigned long long tc_fixed_of(const LdCoreW& ld, int ab, int k, int, int E, uint32_t& sgn) {
    const int r0 = *ld.r0p, bb = ab / r0, a = ab - bb * r0;
    return tc_fixed2(ld.C0[a + (long long)k * ld.ldc], ld.C1w[bb + (long long)k * ld.ldc], E, sgn);
}
FC_DEV unsigned long long tc_fixed_of(const LdKR& ld, int i, int kj, int b, int E, uint32_t& sgn) {
    const int k = kj / ld.S, j = kj - k * ld.S;
    return tc_fixed2(ld.E[b * ld.bsE + i + (long long)k * ld.lde],
                     ld.Y[b * ld.bsY + i + (long long)j * ld.ldy], E, sgn);
}

// Fixed-point values of op(X)[i, k0 + q], q < 8 (zero beyond kend), row i valid.
template <class L>
FC_DEV void tc_fixed_row8(const L& ld, int i, int k0, int kend, int b, int E,
                          unsigned long long (&F)[8], uint32_t (&sg)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        F[q] = 0ull; sg[q] = 0u;
        if (k0 + q < kend) F[q] = tc_fixed_of(ld, i, k0 + q, b, E, sg[q]);
    }
}
FC_DEV void tc_fixed_row8(const LdCoreW& ld, int ab, int k0, int kend, int, int E,
                          unsigned long long (&F)[8], uint32_t (&sg)[8]) {
    const int r0 = *ld.r0p, bb = ab / r0, a = ab - bb * r0;
    const double* p0 = ld.C0 + a;
    const double* p1 = ld.C1w + bb;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        F[q] = 0ull; sg[q] = 0u;
        if (k0 + q < kend)
            F[q] = tc_fixed2(p0[(long long)(k0 + q) * ld.ldc], p1[(long long)(k0 + q) * ld.ldc], E, sg[q]);
    }
}
template <class L>
FC_DEV unsigned long long tc_fixed_of(const TcTrans<L>& t, int j, int k, int b, int E, uint32_t& sg) {
    return tc_fixed_of(t.ld, k, j, b, E, sg);
}

// Exact combination of the level sums v_L (integers |v_L| <= 2^24 held in FP32):
// T = sum_L v_L 2^(7(7-L)) in 128-bit integers (|T| < 2^74), rounded once (to nearest,
// ties away) to FP64 and scaled by 2^(ex - 63).
FC_DEV double tc_combine(const float (&v)[kTcDigits], int ex) {
    long long th = 0, tl = 0;
#pragma unroll
    for (int L = 0; L < 4; ++L) th = th * 128 + (long long)__float2int_rn(v[L]);
#pragma unroll
    for (int L = 4; L < 8; ++L) tl = tl * 128 + (long long)__float2int_rn(v[L]);
    __int128 T = ((__int128)th << 28) + (__int128)tl;
    if (T == 0) return 0.0;
    const bool neg = T < 0;
    unsigned __int128 mag = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    const unsigned long long hi = (unsigned long long)(mag >> 64), lo = (unsigned long long)mag;
    const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);   // bits
    unsigned long long m;
    int e2 = nb - 1;                                  // T = 1.f * 2^e2
    if (nb <= 53) {
        m = lo << (53 - nb);
    } else {
        const int sh = nb - 53;
        unsigned __int128 r = mag >> sh;
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if ((mag & ((half << 1) - 1)) >= half) r += 1;
        if (r >> 53) { r >>= 1; e2 += 1; }
        m = (unsigned long long)r;
    }
    const int ef = e2 + ex - 63 + 1023;               // biased exponent of the result
    if (ef >= 1 && ef <= 2046)
        return __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                                ((unsigned long long)ef << 52) |
                                                (m & 0xFFFFFFFFFFFFFull)));
    const double d = ldexp((double)m, e2 - 52 + ex - 63);      // out of the normal range
    return neg ? -d : d;
}

// f 2^ex as FP64 for a normal or zero FP32 f, by integer operations when in range.
FC_DEV double tc_f2d_scaled(float f, int ex) {
    const uint32_t u = __float_as_uint(f);
    if ((u & 0x7FFFFFFFu) == 0) return 0.0;
    const int e = (int)((u >> 23) & 0xFF) + 896 + ex;
    if (e <= 0 || e >= 2047 || ((u >> 23) & 0xFF) == 0) return ldexp((double)f, ex);
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)e << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// Offset added to F so that plain 7-bit fields of F + kTcOffset are the balanced digits
// plus 64: kTcOffset = 64 sum_{s<8} 2^(56-7s).
constexpr unsigned long long kTcOffset =
    (64ull << 56) | (64ull << 49) | (64ull << 42) | (64ull << 35) | (64ull << 28) |
    (64ull << 21) | (64ull << 14) | (64ull << 7);
// FP32 value of balanced digit s of G = F + kTcOffset with the sign applied:
// ((G >> (56 - 7s)) & 127) - 64 for s > 0, and (G >> 56) - 64 in [0, 64] for the leading
// digit (F < 2^62, so G >> 56 <= 128 carries no further bit), formed as
// (2^23 + u) - (2^23 + 64) (exact) times +-1.  Its BF16 encoding is the upper half of the
// FP32 bits (|d| <= 64: low half zero).
template <int s>
FC_DEV uint32_t tc_digit_f32(unsigned long long G, uint32_t sgn) {
    const uint32_t u = (s == 0) ? (uint32_t)(G >> 56) : ((uint32_t)(G >> (56 - 7 * s)) & 127u);
    const float sf = __uint_as_float(0x3F800000u | sgn);             // +-1
    return __float_as_uint(fmaf(__uint_as_float(0x4B000000u | u), sf, -8388672.0f * sf));
}

FC_DEV void tc_two_sum(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

template <int BN>
struct TcShape {
    static constexpr int PA = kTcBM * kTcKS * 2;            // bytes of one A digit plane
    static constexpr int PB = BN * kTcKS * 2;               // bytes of one B digit plane
    static constexpr int STAGE = kTcDigits * (PA + PB);
    static constexpr int SMEM = 2 * STAGE + 128;            // two stages + alignment slack
    static constexpr int LSTRIDE = (BN <= 16) ? 16 : (BN <= 32) ? 32 : 64;   // TMEM cols / level
    static constexpr int NEED = kTcDigits * LSTRIDE;
    static constexpr int TCOLS = (NEED <= 32) ? 32 : (NEED <= 64) ? 64 : (NEED <= 128) ? 128
                               : (NEED <= 256) ? 256 : 512;
};

// Digits of 8 consecutive K values of one operand row into 16-byte rows of the S planes.
template <int PLANE>
FC_DEV void tc_store8(unsigned char* base, const unsigned long long (&F0)[8], const uint32_t (&sg)[8]) {
    unsigned long long F[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) F[q] = F0[q] + kTcOffset;
#define FC_TC_PLANE(s_)                                                                       \
    {                                                                                         \
        uint32_t w_[4];                                                                       \
        _Pragma("unroll") for (int q = 0; q < 4; ++q)                                         \
            w_[q] = __byte_perm(tc_digit_f32<s_>(F[2 * q], sg[2 * q]),                       \
                                tc_digit_f32<s_>(F[2 * q + 1], sg[2 * q + 1]), 0x7632);       \
        *(uint4*)(base + (s_) * PLANE) = make_uint4(w_[0], w_[1], w_[2], w_[3]);             \
    }
    FC_TC_PLANE(0) FC_TC_PLANE(1) FC_TC_PLANE(2) FC_TC_PLANE(3)
    FC_TC_PLANE(4) FC_TC_PLANE(5) FC_TC_PLANE(6) FC_TC_PLANE(7)
#undef FC_TC_PLANE
}

// Digits of 4 consecutive K values of one operand row: the low or high 8 bytes of a 16-byte
// core-matrix row in each of the S planes.
template <int PLANE>
FC_DEV void tc_store4(unsigned char* base, const unsigned long long (&F0)[4], const uint32_t (&sg)[4]) {
    unsigned long long F[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) F[q] = F0[q] + kTcOffset;
#define FC_TC_PLANE4(s_)                                                                      \
    *(uint2*)(base + (s_) * PLANE) =                                                          \
        make_uint2(__byte_perm(tc_digit_f32<s_>(F[0], sg[0]), tc_digit_f32<s_>(F[1], sg[1]), 0x7632), \
                   __byte_perm(tc_digit_f32<s_>(F[2], sg[2]), tc_digit_f32<s_>(F[3], sg[3]), 0x7632));
    FC_TC_PLANE4(0) FC_TC_PLANE4(1) FC_TC_PLANE4(2) FC_TC_PLANE4(3)
    FC_TC_PLANE4(4) FC_TC_PLANE4(5) FC_TC_PLANE4(6) FC_TC_PLANE4(7)
#undef FC_TC_PLANE4
}

template <int BN, class LA, class LB>
__global__ void __launch_bounds__(kTcBlock, 1)
gemm_tc_kernel(int M, int N, int K, const int* dM, const int* dN, const int* dK,
               LA A, LB B, double alpha, double beta, double* C, int ldc, long long bsC,
               int batch, int splits, int kchunk, unsigned long long* work, int* err,
               int wait_limit)
{
    using Sh = TcShape<BN>;
    constexpr int S = kTcDigits;
    constexpr int NW = kTcThreads / 32;              // producer warps; warp NW issues the MMAs
    constexpr int AQ = kTcThreads / kTcBM;           // threads per row of op(A)
    static_assert(S == 8, "digit planes are unrolled for S = 8");
    static_assert(AQ * 8 == kTcKS, "one 8-wide K group of op(A) per thread and stage");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 64, "MMA N for M = 128");
    static_assert(S * Sh::LSTRIDE <= 512, "TMEM columns");
    extern __shared__ unsigned char tc_dyn[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int s_ea[AQ][kTcBM];
    __shared__ int s_eb[BN];

    if (dM) M = min(M, *dM);
    if (dN) N = min(N, *dN);
    if (dK) K = min(K, *dK);
    const int zb = blockIdx.z / splits, zs = blockIdx.z - zb * splits;
    const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
    if (m0 >= M || n0 >= N || zb >= batch) return;
    const int kbeg = zs * kchunk, kend = min(K, kbeg + kchunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (kTcBM - 1), part = tid / kTcBM;   // op(A) producer: row, K part
    double* Cb = C + zb * bsC;
    if (kend <= kbeg) {                       // empty K range: C = beta C (alone), else nothing
        if (splits == 1 && part == 0 && m0 + row < M)
            for (int j = 0; j < BN && n0 + j < N; ++j) {
                double* c = Cb + (m0 + row) + (long long)(n0 + j) * ldc;
                *c = (beta == 0.0) ? 0.0 : beta * (*c);
            }
        return;
    }
    unsigned char* smem = (unsigned char*)(((uintptr_t)tc_dyn + 127) & ~(uintptr_t)127);

    // ---- scales: row exponents of op(A) (AQ threads per row), column exponents of op(B) --
    const TcTrans<LB> Bt{B};
    if (tid < kTcThreads) {
        const int gi = m0 + row;
        const int kq = (kend - kbeg + AQ - 1) / AQ;
        const int ka = min(kend, kbeg + part * kq), kb = min(kend, ka + kq);
        s_ea[part][row] = (gi < M) ? tc_emax_row(A, gi, ka, kb, zb) : -(1 << 30);
    }
    for (int j = warp; j < BN && warp < NW; j += NW) {
        const int gj = n0 + j;
        int fm = -(1 << 30);
        if (gj < N)
            for (int k = kbeg + lane; k < kend; k += 32) fm = max(fm, tc_ebound(B, k, gj, zb));
        fm = __reduce_max_sync(0xffffffffu, fm);
        if (lane == 0) s_eb[j] = tc_scale_exp(fm);
    }

    // ---- TMEM accumulators and the two stage barriers ------------------------------------
    if (warp == 0) {
        const uint32_t ncols = Sh::TCOLS;
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc_saddr(&s_tmem)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_saddr(&s_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_saddr(&s_bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    int emax = s_ea[0][row];
#pragma unroll
    for (int q = 1; q < AQ; ++q) emax = max(emax, s_ea[q][row]);
    const int Ea = tc_scale_exp(emax);

    const uint32_t idesc = (1u << 4)                        // D: FP32
                         | (1u << 7) | (1u << 10)           // A, B: BF16 (K-major)
                         | ((uint32_t)(BN >> 3) << 17)      // N / 8
                         | ((uint32_t)(kTcBM >> 4) << 24);  // M / 16
    // Pipeline: producers fill stage st of buffer st & 1 once the MMAs of stage st - 2 (which
    // read that buffer) have completed: one lane per warp waits on the buffer's mbarrier.  The
    // MMA warp issues stage st after the block barrier and commits it to the same mbarrier, so
    // the issue overlaps the production of stage st + 1.  The commit of stage t is the
    // (t >> 1)-th completion of barrier t & 1: its phase parity is (t >> 1) & 1.  A failed
    // wait ends the loop in every thread at the next barrier (__syncthreads_or).
    const int nst = (kend - kbeg + kTcKS - 1) / kTcKS;
    const bool producer = tid < kTcThreads;
    int issued = 0;                                   // stages issued (MMA thread)
    bool bad = false;
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        unsigned char* sa = smem + buf * Sh::STAGE;
        unsigned char* sb = sa + S * Sh::PA;
        if (producer) {
            if (st >= 2) {
                int ok = 1;
                if (lane == 0)
                    ok = tc_wait(tc_saddr(&s_bar[buf]), (uint32_t)(((st - 2) >> 1) & 1), wait_limit) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp();                         // the warp's writes follow the wait
                bad = (ok == 0);
            }
            if (!bad) {
                const int k0 = kbeg + st * kTcKS;
                // op(A) digits: thread <-> (row, 8-wide K group = one 16-byte core-matrix row)
                {
                    const int gi = m0 + row;
                    unsigned long long F[8];
                    uint32_t sg[8];
                    if (gi < M) tc_fixed_row8(A, gi, k0 + part * 8, kend, zb, Ea, F, sg);
                    else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) { F[q] = 0ull; sg[q] = 0u; }
                    }
                    tc_store8<Sh::PA>(sa + (row & 7) * 16 + (row >> 3) * 512 + part * 128, F, sg);
                }
                // op(B) digits: thread <-> (column j, 4-wide K group), 8-byte stores; the
                // half-width groups spread B over twice as many warps
                for (int task = tid; task < BN * (kTcKS / 4); task += kTcThreads) {
                    const int j = task % BN, h = task / BN, gj = n0 + j;
                    unsigned long long F[4];
                    uint32_t sg[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        F[q] = 0ull; sg[q] = 0u;
                        const int k = k0 + h * 4 + q;
                        if (gj < N && k < kend) F[q] = tc_fixed_of(Bt, gj, k, zb, s_eb[j], sg[q]);
                    }
                    tc_store4<Sh::PB>(sb + (j & 7) * 16 + (j >> 3) * 512 + (h >> 1) * 128 + (h & 1) * 8,
                                      F, sg);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        if (__syncthreads_or(bad ? 1 : 0)) { bad = true; break; }
        if (tid == kTcThreads) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = tc_saddr(sa), b0 = tc_saddr(sb);
#pragma unroll 1
            for (int L = 0; L < S; ++L)
#pragma unroll 1
                for (int s = 0; s <= L; ++s)
#pragma unroll
                    for (int ks = 0; ks < kTcKS / 16; ++ks) {
                        const uint64_t da = tc_desc(a0 + s * Sh::PA + ks * 256, 128, 512);
                        const uint64_t db = tc_desc(b0 + (L - s) * Sh::PB + ks * 256, 128, 512);
                        const uint32_t acc = (st > 0 || s > 0 || ks > 0) ? 1u : 0u;
                        tc_mma(tmem + (uint32_t)(L * Sh::LSTRIDE), da, db, idesc, acc);
                    }
            tc_commit(tc_saddr(&s_bar[buf]));
            issued = st + 1;
        }
    }
    // ---- epilogue: wait for the last commit, combine the levels, add to C ----------------
    {
        int fail = bad ? 1 : 0;
        if (!bad && tid == kTcThreads)
            fail = tc_wait(tc_saddr(&s_bar[(nst - 1) & 1]), (uint32_t)(((nst - 1) >> 1) & 1)) ? 0 : 1;
        if (bad && tid == kTcThreads && issued > 0)   // drain what was issued before freeing TMEM
            (void)tc_wait(tc_saddr(&s_bar[(issued - 1) & 1]), (uint32_t)(((issued - 1) >> 1) & 1));
        bad = __syncthreads_or(fail) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!bad && producer) {
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (rows) and the 8-column chunks
        // w / 4, w / 4 + NW / 4, ... of the tile
        const int q4 = warp & 3;
        const int r = q4 * 32 + lane, gi = m0 + r;
        int em = s_ea[0][r];
#pragma unroll
        for (int q = 1; q < AQ; ++q) em = max(em, s_ea[q][r]);
        const int Ei = tc_scale_exp(em);
        const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
#pragma unroll 1
        for (int j0 = (warp >> 2) * 8; j0 < BN; j0 += (NW / 4) * 8) {
            float lv[S][8];
#pragma unroll
            for (int L = 0; L < S; ++L) tc_ld8(tl + (uint32_t)(L * Sh::LSTRIDE + j0), lv[L]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (gi >= M) continue;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int gj = n0 + j0 + jj;
                if (gj >= N) continue;
                const int Eb = s_eb[j0 + jj];
                double v;
                if (Ei == kTcBadExp || Eb == kTcBadExp) {
                    v = __longlong_as_double(0x7ff8000000000000ll);
                } else {
                    float col[S];
#pragma unroll
                    for (int L = 0; L < S; ++L) col[L] = lv[L][jj];
                    v = tc_combine(col, Ei + Eb);
                }
                if (alpha != 1.0) v *= alpha;
                double* c = Cb + gi + (long long)gj * ldc;
                if (splits > 1) atomicAdd(c, v);
                else *c = (beta == 0.0) ? v : v + beta * (*c);
            }
        }
        // instrumentation: BF16 MMA flops issued by this CTA (36 digit pairs per K step)
        if (work && tid == 0)
            atomicAdd(work, (unsigned long long)(S * (S + 1) / 2) * 2ull * kTcBM * BN *
                                (unsigned long long)(nst * kTcKS));
    } else if (bad && tid == 0) {
        atomicExch(err ? err : &g_tc_error, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        const uint32_t ncols = Sh::TCOLS;
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols) : "memory");
    }
}

// Per-device one-time opt-in of an instantiation to its dynamic shared memory.
template <int BN, class LA, class LB>
inline bool tc_prepare() {
    static int done[16] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return false;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(gemm_tc_kernel<BN, LA, LB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcShape<BN>::SMEM) != cudaSuccess)
            return false;
        done[dev] = 1;
    }
    return true;
}

// Launch: N tile of 16/32/48/64 and K ranges of at most kTcKC.  Returns false if the
// instantiation could not be prepared (nothing launched).
template <class LA, class LB>
inline bool gemm_tc(cudaStream_t st, int M, int N, int K, LA A, LB B, double alpha, double beta,
                    double* C, int ldc, long long bsC, int batch, const int* dM, const int* dN,
                    const int* dK)
{
    if (M <= 0 || N <= 0 || batch <= 0) return true;
    const int BN = (N <= 16) ? 16 : (N <= 32) ? 32 : (N <= 48) ? 48 : 64;
    const long long tiles = (long long)((M + kTcBM - 1) / kTcBM) * ((N + BN - 1) / BN) * batch;
    // fewest K ranges of at most kTcKC, then (schedule field tc_split) as many as fill the
    // waves of one CTA per SM (at least 64 of K each)
    const int smin = std::max(1, (K + kTcKC - 1) / kTcKC);
    const long long waves = (tiles * smin + kNumSMs - 1) / kNumSMs;
    int splits = smin;
    if (sched(g_sched.tc_split))
        splits = (int)std::max<long long>(
            smin, std::min<long long>(waves * kNumSMs / tiles, std::max(1, (K + 63) / 64)));
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + kTcKS - 1) / kTcKS * kTcKS;
    if (kchunk > kTcKC) kchunk = kTcKC;
    if (kchunk < kTcKS) kchunk = kTcKS;
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    bool ok;
    switch (BN) {
        case 16: ok = tc_prepare<16, LA, LB>(); break;
        case 32: ok = tc_prepare<32, LA, LB>(); break;
        case 48: ok = tc_prepare<48, LA, LB>(); break;
        default: ok = tc_prepare<64, LA, LB>(); break;
    }
    if (!ok) return false;
    if (splits > 1 && beta != 1.0) {
        dim3 g((M + 255) / 256, N, batch);
        note_launch(); gemm_prescale_kernel<<<g, 256, 0, st>>>(M, N, dM, dN, beta, C, ldc, bsC);
    }
    dim3 grid((M + kTcBM - 1) / kTcBM, (N + BN - 1) / BN, batch * splits);
    const bool prof = prof_active(KC_TC);
    unsigned long long* work = prof ? prof_work_counter() : nullptr;
    int* err = tc_error_target();
    const int wl = tc_producer_wait_limit();
    ProfMark mark;
    if (prof) prof_begin(st, mark);
    note_launch();
    switch (BN) {
        case 16:
            gemm_tc_kernel<16, LA, LB><<<grid, kTcBlock, TcShape<16>::SMEM, st>>>(
                M, N, K, dM, dN, dK, A, B, alpha, beta, C, ldc, bsC, batch, splits, kchunk, work, err, wl);
            break;
        case 32:
            gemm_tc_kernel<32, LA, LB><<<grid, kTcBlock, TcShape<32>::SMEM, st>>>(
                M, N, K, dM, dN, dK, A, B, alpha, beta, C, ldc, bsC, batch, splits, kchunk, work, err, wl);
            break;
        case 48:
            gemm_tc_kernel<48, LA, LB><<<grid, kTcBlock, TcShape<48>::SMEM, st>>>(
                M, N, K, dM, dN, dK, A, B, alpha, beta, C, ldc, bsC, batch, splits, kchunk, work, err, wl);
            break;
        default:
            gemm_tc_kernel<64, LA, LB><<<grid, kTcBlock, TcShape<64>::SMEM, st>>>(
                M, N, K, dM, dN, dK, A, B, alpha, beta, C, ldc, bsC, batch, splits, kchunk, work, err, wl);
            break;
    }
    if (prof) prof_end(st, mark);
    return true;
}

}  // namespace fc
