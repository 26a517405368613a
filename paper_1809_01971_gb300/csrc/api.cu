// libfc C ABI: handle, setup, workspace, and the host orchestration of the low-rank PCG
// (Algorithm 1 of Section 3.3) over the device kernels.  Every arithmetic step of the
// path runs in device kernels; the host only sequences launches, reads back ranks and
// the FP64 PCG scalars.
#include "../../include/fc.h"
#include "fc_common.cuh"
#include "fc_kernels.h"
#include "setup_host.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

using namespace fc;

#include <atomic>

namespace fc {
SchedState g_sched;
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Tensor-core error flag of the calling thread's current handle call (a slot of that
// handle's workspace; null outside handle calls) and the producer-side wait limit.
static thread_local int* t_tc_flag = nullptr;
static std::atomic<int> g_tc_wait_limit{kTcWaitFull};
int* tc_error_target() { return t_tc_flag; }
int tc_producer_wait_limit() { return g_tc_wait_limit.load(std::memory_order_relaxed); }

// Instrumentation state: one enabled kernel class, a growing pool of event pairs.
static std::mutex g_prof_mu;
static std::atomic<int> g_prof_class{KC_NONE};
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_events;
static size_t g_prof_used = 0;

bool prof_active(int kclass) { return g_prof_class.load(std::memory_order_relaxed) == kclass; }

void prof_begin(cudaStream_t st, ProfMark& m) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (g_prof_used == g_prof_events.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
        g_prof_events.emplace_back(a, b);
    }
    m.slot = (int)g_prof_used++;
    cudaEventRecord(g_prof_events[m.slot].first, st);
}

void prof_end(cudaStream_t st, const ProfMark& m) {
    if (m.slot < 0) return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    cudaEventRecord(g_prof_events[m.slot].second, st);
}
}  // namespace fc

namespace {

thread_local std::string g_cuda_msg;

int cuda_fail(cudaError_t e) {
    g_cuda_msg = cudaGetErrorString(e);
    return FC_ECUDA;
}
}  // namespace

int fc::record_cuda_error(cudaError_t e) { return cuda_fail(e); }

namespace {
#define CK(x)                                        \
    do {                                             \
        cudaError_t _e = (x);                        \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)
#define CKL()                                                 \
    do {                                                      \
        cudaError_t _e = cudaGetLastError();                  \
        if (_e != cudaSuccess) return cuda_fail(_e);          \
    } while (0)

// Internal CP tensor: factor matrices of one tensor are contiguous, mode stride = ld * cap.
struct CP {
    int rank = 0, cap = 0, ld = 0;
    double* xi = nullptr;
    double* U[3] = {nullptr, nullptr, nullptr};
    long long bs() const { return (long long)ld * cap; }
};

// Fraction of a truncation budget below which the eigen-solves leave an off-diagonal entry
// unrotated (launch_gjacobi's absolute floor).
constexpr double kEnergyFloor = 0.01;

// Linear bump allocator over the caller's workspace (256-byte aligned slices).
struct Arena {
    char* base = nullptr;
    size_t off = 0, cap = 0;
    bool count_only = true;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = count_only ? nullptr : base + off;
        off += bytes;
        return p;
    }
    double* d(size_t count) { return (double*)take(count * sizeof(double)); }
    int* i(size_t count) { return (int*)take(count * sizeof(int)); }
};

}  // namespace

struct fc_ctx {
    int n = 0, d = 0;
    double alpha = 0, beta = 0, gamma = 0, eps = 0;
    fc_setup_opts opts{};
    fc_setup_info info{};
    int RA = 0, RP = 0;   // symbol / preconditioner ranks
    int CAP = 0;          // CP rank cap of the iterates
    int KIN = 0;          // largest input rank of apply/precond/truncate
    int RM = 0;           // max Tucker rank
    int CM = kMaxC;       // sketch width
    int QMAX = 0;         // largest output rank of a truncation
    long long KMAX = 0;   // largest number of terms entering a truncation
    // device tables (owned)
    double* tables = nullptr;
    double *lam = nullptr, *sintab = nullptr;
    double *xiA = nullptr, *EA = nullptr;   // symbol CP (weights, unit-column mode factors)
    double *xiP = nullptr, *EP = nullptr;   // preconditioner CP
    // state symbol beta rho^-alpha: the first RS columns of EA with weights xiA / beta
    double *xiS = nullptr;
    // dominating column weights of the three symbols' Khatri-Rao side matrices, per mode
    // (mode stride R): xw_l[k] = |xi_k| prod_{m != l} max_i |E_m[i, k]| (see symbol_proxy_weights)
    double *xiAw = nullptr, *xiPw = nullptr, *xiSw = nullptr;
    int RS = 0;
    SymbolSpec spec;      // operator symbol g(rho) = a rho^-sn + b rho^sp + c
    bool spectral = false;   // during a spectral-resident solve: operands already in the eigenbasis
    double* V = nullptr;     // variable coefficients: orthonormal eigenvector matrices of the 1D
                             // stiffness matrices (d x n x n, column-major), else the DST-I
    double alpha_eff = 0.0;   // exponent of the symbol's spectrum (1 for the directional operator)
    double2* twid = nullptr;  // e^{-i pi k / (n+1)}, k <= n (fast sine transforms; n+1 a power of
                              // two, n < 4096)
    int prec = GP_F64;        // contractions in FP64 or double-float FP32 (fc_setup_opts.precision)
    // compressed mode factors of the three symbols (operator, preconditioner, state):
    // Et[s] (3 modes x n x rE[s]) and Mt[s] (3 modes x rE[s] x R_s), see compress_factor
    double* ctab = nullptr;
    double *Et[3] = {nullptr, nullptr, nullptr}, *Mt[3] = {nullptr, nullptr, nullptr};
    int rE[3] = {0, 0, 0};
    int rEmax = 0;
    // workspace (caller-owned)
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // workspace slices
    struct {
        double *Y, *Y2, *Q, *tmp, *M, *Tm, *GQ, *Tr, *theta, *Vr, *Z, *Zr, *C, *Cq, *wK, *C2, *wN;
        double *core, *G3, *ev3, *W3, *Srot, *SG, *mus, *Vs, *sigma, *X, *Yh, *Nu;
        double *scal, *Mi;
        int *dims, *tslice, *tidx;
        CP cat, Xs, Rs, Ps, Zs, Ss, Xb;
        double* pinned_dummy;
    } w{};
    static constexpr unsigned long long kSeed0 = 0x1809019710ull;
    unsigned long long seed = kSeed0;
    // rank statistics of the truncations since the last reset (fc_solve reports them)
    long long stat_rsum = 0, stat_rcount = 0;
    int stat_rmax = 0, stat_bmax = 0;
    // host pinned scalars for readback
    double* hbuf = nullptr;
    int* hint = nullptr;
};

namespace {

size_t layout(fc_ctx* h, Arena& a) {
    const int n = h->n, d = h->d, CM = h->CM, RM = h->RM;
    const long long K = h->KMAX;
    auto& w = h->w;
    const size_t nC = (size_t)n * CM;
    w.Y = a.d(3 * nC);
    w.Y2 = a.d(3 * nC);
    w.Q = a.d(3 * nC);
    w.tmp = a.d(3 * nC);
    w.M = a.d(3 * (size_t)CM * CM);
    w.Tm = a.d(3 * (size_t)CM * CM);
    w.GQ = a.d(3 * nC);
    w.Tr = a.d(3 * (size_t)CM * CM);
    w.theta = a.d(3 * (size_t)CM);
    w.Vr = a.d(3 * (size_t)CM * CM);
    w.Z = a.d(3 * nC);
    w.Zr = a.d(3 * nC);
    w.C = a.d(3 * (size_t)std::max(RM, CM) * K);
    w.Cq = a.d(3 * (size_t)CM * K);
    w.wK = a.d((size_t)K);
    w.C2 = a.d(3 * (size_t)CM * std::max<long long>(1, (long long)h->rEmax * h->KIN));
    w.wN = a.d(3 * (size_t)K);
    w.core = a.d((size_t)RM * RM * RM);
    w.G3 = a.d((size_t)RM * RM);
    w.ev3 = a.d((size_t)RM);
    w.W3 = a.d((size_t)RM * RM);
    w.Srot = a.d((size_t)RM * RM * RM);
    w.SG = a.d((size_t)RM * RM * RM);
    w.mus = a.d((size_t)RM * RM);
    w.Vs = a.d((size_t)RM * RM * RM);
    w.sigma = a.d((size_t)RM * RM);
    w.X = a.d(3 * (size_t)RM * h->QMAX);
    w.Yh = a.d(3 * (size_t)n * h->KIN);
    w.Nu = a.d(3 * (size_t)std::max(h->RA, h->RP) * h->KIN);
    w.scal = a.d(64);
    w.Mi = a.d(3 * (size_t)h->KIN * h->KIN);
    w.dims = a.i(D_SIZE);
    w.tslice = a.i((size_t)RM * RM);
    w.tidx = a.i((size_t)RM * RM);
    auto mkcp = [&](CP& c, int cap) {
        c.cap = cap; c.ld = n; c.rank = 0;
        c.xi = a.d(cap);
        double* U = a.d((size_t)3 * n * cap);
        for (int l = 0; l < 3; ++l) c.U[l] = U ? U + (size_t)l * n * cap : nullptr;
    };
    mkcp(w.cat, std::max(2 * h->CAP, h->KIN));
    mkcp(w.Xs, h->CAP);
    mkcp(w.Rs, std::max(h->CAP, h->KIN));
    mkcp(w.Ps, h->CAP);
    mkcp(w.Zs, h->CAP);
    mkcp(w.Ss, h->CAP);
    mkcp(w.Xb, h->CAP);
    (void)d;
    return a.off + 256;
}

// Kernel attributes are per device: set them once for every device the library runs on.
int ensure_attributes() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FC_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        cudaError_t e = set_linalg_attributes();
        if (e == cudaSuccess) e = set_symeig_attributes();
        if (e == cudaSuccess) e = set_fft_attributes(4096);   // the largest line length
        if (e != cudaSuccess) return cuda_fail(e);
        done[dev] = true;
    }
    return FC_OK;
}

// Compressed mode factors of the operator, preconditioner and state symbols (cold path):
// the factors built on the device are read back, compressed on the host in FP64
// (compress_factor, relative tolerance kCompressTol per spectral row) and uploaded as Et / Mt.
// Relative tolerance of the compressed symbol factors (per spectral row): at n = 8191 and
// alpha = 0.75 a looser 1e-12 left 5e-7 in the solution of a sine-mode right-hand side.
constexpr double kCompressTol = 1e-14;

// Dominating weights of a symbol's Khatri-Rao side matrices (cold path, host).  A mat-vec
// output has the terms xa_k xb_j (x)_l (e_lk . y_lj) with unit e_lk, y_lj; its columns are not
// unit vectors (nu_l(k, j) = ||e_lk . y_lj|| <= ||e_lk||_inf), so the column-normalised tensor
// has the weights |xa_k xb_j| prod_l nu_l(k, j).  The stage-1 sketch of mode l is taken with
// the columns e_lk . y_lj and the weights |xa_k xb_j| prod_{m != l} ||e_mk||_inf, which dominate
// the normalised weights column by column, so the energy it leaves outside its basis bounds
// the normalised one, while the weights keep the Khatri-Rao product form (xa_k-part times xb_j)
// that the structured sketch and the compressed symbol factors need.
int symbol_proxy_weights(fc_ctx* h) {
    const int n = h->n, d = h->d;
    const int Rs[3] = {h->RA, h->RP, h->RS};
    const double* Edev[3] = {h->EA, h->EP, h->EA};
    const long long bsE[3] = {(long long)n * h->RA, (long long)n * h->RP, (long long)n * h->RA};
    const double* xdev[3] = {h->xiA, h->xiP, h->xiS};
    double* out[3] = {h->xiAw, h->xiPw, h->xiSw};
    for (int sy = 0; sy < 3; ++sy) {
        const int R = Rs[sy];
        if (R == 0) continue;
        std::vector<double> E((size_t)n * R), xa(R), cmax((size_t)3 * R, 1.0), xw((size_t)3 * R, 0.0);
        CK(cudaMemcpy(xa.data(), xdev[sy], sizeof(double) * R, cudaMemcpyDeviceToHost));
        for (int l = 0; l < d; ++l) {
            CK(cudaMemcpy(E.data(), Edev[sy] + l * bsE[sy], sizeof(double) * n * R,
                          cudaMemcpyDeviceToHost));
            for (int k = 0; k < R; ++k) {
                double m = 0.0;
                for (int i = 0; i < n; ++i) m = std::max(m, std::fabs(E[i + (size_t)k * n]));
                cmax[(size_t)l * R + k] = m;
            }
        }
        for (int l = 0; l < d; ++l)
            for (int k = 0; k < R; ++k) {
                double v = std::fabs(xa[k]);
                for (int m = 0; m < d; ++m)
                    if (m != l) v *= cmax[(size_t)m * R + k];
                xw[(size_t)l * R + k] = v;
            }
        CK(cudaMemcpy(out[sy], xw.data(), sizeof(double) * 3 * R, cudaMemcpyHostToDevice));
    }
    return FC_OK;
}

int compress_symbols(fc_ctx* h) {
    const int n = h->n, d = h->d;
    const int Rs[3] = {h->RA, h->RP, h->RS};
    const double* Edev[3] = {h->EA, h->EP, h->EA};
    const long long bsE[3] = {(long long)n * h->RA, (long long)n * h->RP, (long long)n * h->RA};
    const double* xdev[3] = {h->xiAw, h->xiPw, h->xiSw};   // per-mode dominating weights
    std::vector<Compressed> comp(3 * d);
    for (int sy = 0; sy < 3; ++sy) {
        const int R = Rs[sy];
        if (R == 0) continue;                 // no state symbol for the test operators
        std::vector<double> E((size_t)n * R), xa(R);
        for (int l = 0; l < d; ++l) {
            CK(cudaMemcpy(xa.data(), xdev[sy] + (size_t)l * R, sizeof(double) * R,
                          cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(E.data(), Edev[sy] + l * bsE[sy], sizeof(double) * n * R,
                          cudaMemcpyDeviceToHost));
            if (!compress_factor(E.data(), n, R, xa.data(), kCompressTol, comp[sy * d + l]))
                return FC_ESETUP;
        }
    }
    size_t total = 0;
    for (int sy = 0; sy < 3; ++sy) {
        int r = 0;
        for (int l = 0; l < d; ++l) r = std::max(r, comp[sy * d + l].r);
        h->rE[sy] = r;
        h->rEmax = std::max(h->rEmax, r);
        total += 3 * ((size_t)n * r + (size_t)r * Rs[sy]);
    }

    if (cudaMalloc(&h->ctab, total * sizeof(double)) != cudaSuccess) return FC_ECUDA;
    CK(cudaMemset(h->ctab, 0, total * sizeof(double)));
    double* p = h->ctab;
    for (int sy = 0; sy < 3; ++sy) {
        const int r = h->rE[sy], R = Rs[sy];
        h->Et[sy] = p; p += 3 * (size_t)n * r;
        h->Mt[sy] = p; p += 3 * (size_t)r * R;
        for (int l = 0; l < d; ++l) {
            const Compressed& c = comp[sy * d + l];   // zero-padded to r columns / rows
            std::vector<double> Et((size_t)n * r, 0.0), Mt((size_t)r * R, 0.0);
            for (int a = 0; a < c.r; ++a)
                for (int i = 0; i < n; ++i) Et[i + (size_t)a * n] = c.Et[i + (size_t)a * n];
            for (int k = 0; k < R; ++k)
                for (int a = 0; a < c.r; ++a) Mt[a + (size_t)k * r] = c.Mt[a + (size_t)k * c.r];
            CK(cudaMemcpy(h->Et[sy] + (size_t)l * n * r, Et.data(), sizeof(double) * n * r,
                          cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->Mt[sy] + (size_t)l * r * R, Mt.data(), sizeof(double) * r * R,
                          cudaMemcpyHostToDevice));
        }
    }
    return FC_OK;
}

CP from_user(const fc_cp* x) {
    CP c;
    c.rank = x->rank; c.cap = x->cap; c.ld = x->ld; c.xi = x->xi;
    for (int l = 0; l < 3; ++l) c.U[l] = x->U[l];
    return c;
}

bool check_cp(const fc_ctx* h, const fc_cp* x, bool output) {
    if (!x) return false;
    if (x->d != h->d || x->n != h->n || x->ld < h->n || x->cap < 0) return false;
    if (!output && (x->rank < 0 || x->rank > x->cap)) return false;
    if (x->cap > 0 && (!x->xi || !x->U[0] || !x->U[1] || (h->d == 3 && !x->U[2]))) return false;
    return true;
}

// Mode-wise transform to the operator's eigenbasis and back, on `cols` columns of every mode:
// the DST-I out_l = F in_l for the Laplacian (Section 3.2, F = F^T = F^{-1}); with per-mode
// eigenbases V_l (variable coefficients), out_l = V_l^T in_l forward and V_l in_l back.
void eig_transform_cols(fc_ctx* h, cudaStream_t st, int cols, const double* const in[3], int ldi,
              double* const out[3], int ldo, bool forward) {
    if (cols <= 0) return;
    const int n = h->n;
    if (h->V) {             // per-mode eigenbases: forward V_l^T x, inverse V_l x
        for (int l = 0; l < h->d; ++l) {
            const double* Vl = h->V + (long long)l * n * n;
            if (forward)
                gemm_p(h->prec, st, n, cols, n, LdT{Vl, n, 0}, LdN{in[l], ldi, 0}, 1.0, 0.0, out[l], ldo);
            else
                gemm_p(h->prec, st, n, cols, n, LdN{Vl, n, 0}, LdN{in[l], ldi, 0}, 1.0, 0.0, out[l], ldo);
        }
        return;
    }
    LdSine F{h->sintab, 2 * (n + 1)};
    for (int l = 0; l < h->d; ++l)
        gemm_p(h->prec, st, n, cols, n, F, LdN{in[l], ldi, 0}, 1.0, 0.0, out[l], ldo);
}

struct KRIn {           // implicit Khatri-Rao tensor sum_{k,j} xa_k xb_j (x)_l E_l[:,k].Yh_l[:,j]
    const double* xa; const double* E; int Ra; long long bsE;
    const double* xb; const double* Yh; int S;
    // compressed symbol factors E_l ~ Et_l Mt_l (Et_l: n x rE, Mt_l: rE x Ra, mode strides
    // bsEt, bsMt); Et_l has the same Gram as E_l diag|xa|, so the Khatri-Rao tensor's side
    // matrices have the same Gram as those of Et_l . (Yh_l diag|xb|) with rE * S columns
    const double* Et; long long bsEt; const double* Mt; long long bsMt; int rE;
};
struct DenseIn { const double* w; const double* U; int ld; long long bs; int K; };

// The tensor-core GEMMs of a handle call record an expired bounded wait in the flag slot
// dims[D_FLAG] of the handle's workspace (HandleCall points the launches there and clears it
// at entry).  The slot travels to the host with the truncation's dims copy (h->hint); calls
// without a truncation copy it themselves (flag_to_host) before their synchronisation.
int tc_status(const fc_ctx* h) { return h->hint[D_FLAG] ? FC_ETIMEOUT : FC_OK; }

int flag_to_host(fc_ctx* h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->hint + D_FLAG, h->w.dims + D_FLAG, sizeof(int), cudaMemcpyDeviceToHost, st));
    return FC_OK;
}

// Scope of one API call on a handle: the calling thread's tensor-core launches report into
// the handle's flag slot, which starts cleared; the contraction form may be overridden.
struct HandleCall {
    fc_ctx* h;
    int* prev_flag;
    int prev_prec;
    int rc = FC_OK;
    HandleCall(fc_ctx* h_, cudaStream_t st, int prec_override = -1)
        : h(h_), prev_flag(t_tc_flag), prev_prec(h_->prec) {
        t_tc_flag = h->w.dims + D_FLAG;
        h->hint[D_FLAG] = 0;
        if (prec_override >= 0) h->prec = prec_override;
        cudaError_t e = cudaMemsetAsync(h->w.dims + D_FLAG, 0, sizeof(int), st);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    ~HandleCall() {
        t_tc_flag = prev_flag;
        h->prec = prev_prec;
    }
};

// ---------------------------------------------------------------------------------------
// Truncation (Section 5, RHOSVD canonical -> Tucker -> canonical).  Input either an
// implicit Khatri-Rao tensor in the eigen-index domain (mat-vec outputs; the Tucker bases
// are transformed back with one DST of their r_l columns) or explicit factors.  Output
// written to `out` (rank set after a stream synchronisation).
// ---------------------------------------------------------------------------------------
int truncate_impl(fc_ctx* h, cudaStream_t st, const KRIn* kr, const DenseIn* dn, double eps,
                  int maxq, CP& out) {
    auto& w = h->w;
    const int n = h->n, d = h->d, CM = h->CM, RM = h->RM;
    const long long nC = (long long)n * CM;
    const long long K = kr ? (long long)kr->Ra * kr->S : dn->K;
    if (K <= 0) { out.rank = 0; return FC_OK; }
    if (K > h->KMAX) return FC_ERANK;
    maxq = std::min(maxq, std::min(out.cap, h->QMAX));
    // Stage 1 sees the side matrices through a matrix with the same Gram: the explicit
    // columns, or for a mat-vec output the compressed Khatri-Rao matrix (Kt = rE * S columns).
    const long long Kt = kr ? (long long)kr->rE * kr->S : K;
    // Sketch: Kt <= CM explicit columns (c = cs = Kt); otherwise CM random columns, of which
    // the first cs = CM - kHold span the basis and the last kHold estimate the energy it misses.
    const bool sketch = Kt > CM;
    const int c = sketch ? CM : (int)Kt;
    const int cs = sketch ? CM - kHold : c;
    const unsigned long long seed = (h->seed += 0x9E3779B97F4A7C15ull);
    // contraction form of the n-sized products of the truncation (sketches, Cholesky-QR Grams
    // and bases, the Ritz basis, the output factors): the tensor-core digits in form 3, FP64
    // otherwise (the orthonormalisation needs FP64-accurate Grams, which double-float is not)
    const int bp = (h->prec == GP_TC64) ? GP_TC64 : GP_F64;
    int* dims = w.dims;
    CK(cudaMemsetAsync(dims, 0, sizeof(int) * D_FLAG, st));
    CK(cudaMemsetAsync(w.scal, 0, sizeof(double) * 64, st));

    // ---- stage 1: range of the weighted side matrices W_l = U_l diag|w| ------------------
    if (kr) {
        if (!sketch)
            launch_kr_cols(st, d, n, kr->rE, kr->S, kr->Et, n, kr->bsEt, nullptr,
                           kr->Yh, n, (long long)n * h->KIN, kr->xb, 1, w.Y, n, nC);
        else
            launch_sketch_kr(st, bp, d, n, kr->rE, kr->S, c, kr->Et, n, kr->bsEt, nullptr,
                             kr->Yh, n, (long long)n * h->KIN, kr->xb, seed, w.Y, n, nC, w.tmp);
    } else {
        if (!sketch)
            launch_scale_cols_abs(st, d, n, (int)K, dn->U, dn->ld, dn->bs, dn->w, w.Y, n, nC);
        else
            launch_sketch_dense(st, bp, d, n, (int)K, c, dn->U, dn->ld, dn->bs, dn->w, seed, w.Y, n, nC);
    }
    CKL();
    // Orthonormal basis of range(Y[:, :cs]) by pivoted Cholesky-QR with one deflation level.
    // A Cholesky factor of the Gram resolves only directions with sigma / sigma_max above
    // ~sqrt(relTol) = 3e-8; the directions it drops are recovered from the remainder
    // Y - Q1 Q1^T Y, which is column-normalised and orthonormalised on its own, then
    // appended to Q1 and re-orthonormalised (span preserved to ~1e-15 relative).
    const long long CC = (long long)CM * CM;
    auto cholqr = [&](const double* src, double* dst, int* rk) {
        gemm_p(bp, st, cs, cs, n, LdT{src, n, nC}, LdN{src, n, nC}, 1.0, 0.0, w.M, CM, CC, d);
        launch_pchol(st, d, w.M, CM, CC, nullptr, 0, cs, 1e-15, w.Tm, CM, CC, rk, 1);
        gemm_p(bp, st, n, cs, cs, LdN{src, n, nC}, LdN{w.Tm, CM, CC}, 1.0, 0.0, dst, n, nC, d);
    };
    cholqr(w.Y, w.Q, dims + D_C1);           // Q1 (orthogonal to ~kappa^2 u)
    cholqr(w.Q, w.Y2, dims + D_C1);          // Q1 re-orthonormalised
    // remainder tmp = Y - Q1 (Q1^T Y), columns scaled to unit norm (zero if at rounding level)
    gemm_p(bp, st, cs, cs, n, LdT{w.Y2, n, nC}, LdN{w.Y, n, nC}, 1.0, 0.0, w.Tr, CM, CC, d);
    CK(cudaMemcpyAsync(w.tmp, w.Y, sizeof(double) * d * nC, cudaMemcpyDeviceToDevice, st));
    gemm_p(bp, st, n, cs, cs, LdN{w.Y2, n, nC}, LdN{w.Tr, CM, CC}, -1.0, 1.0, w.tmp, n, nC, d);
    launch_deflate_normalize(st, d, n, cs, w.tmp, n, nC, w.Y, 1e-13);
    cholqr(w.tmp, w.Q, dims + D_CR);         // Q2
    // Q2 <- Q2 - Q1 (Q1^T Q2), re-orthonormalised
    gemm_p(bp, st, cs, cs, n, LdT{w.Y2, n, nC}, LdN{w.Q, n, nC}, 1.0, 0.0, w.Tr, CM, CC, d);
    gemm_p(bp, st, n, cs, cs, LdN{w.Y2, n, nC}, LdN{w.Tr, CM, CC}, -1.0, 1.0, w.Q, n, nC, d);
    cholqr(w.Q, w.GQ, dims + D_CR);
    // [Q1 | Q2] and a final pass; live columns of the basis -> dims[D_C1 + l]
    launch_combine_cols(st, d, n, cs, w.Y2, n, nC, w.GQ, dims + D_C1, dims + D_CR, dims + D_CT);
    cholqr(w.Y2, w.Q, dims + D_C1);
    double* Qb = w.Q;
    CKL();
    // Energy the basis misses, (1/kHold) ||(I - Q Q^T) Y_hold||_F^2 (an unbiased estimate of
    // ||(I - Q Q^T) W||_F^2 for sketch columns W omega with E[omega omega^T] = I); computed
    // from the projected residual itself, so it is resolved down to rounding level.
    if (sketch) {
        double* Yh = w.Y + (long long)cs * n;
        double* Rh = w.tmp + (long long)cs * n;
        gemm(st, cs, kHold, n, LdT{Qb, n, nC}, LdN{Yh, n, nC}, 1.0, 0.0, w.Tr, CM, CC, d);
        CK(cudaMemcpy2DAsync(Rh, sizeof(double) * nC, Yh, sizeof(double) * nC,
                             sizeof(double) * n * kHold, d, cudaMemcpyDeviceToDevice, st));
        gemm(st, n, kHold, cs, LdN{Qb, n, nC}, LdN{w.Tr, CM, CC}, -1.0, 1.0, Rh, n, nC, d);
        launch_block_energy(st, d, n * kHold, Rh, nC, 1.0 / kHold, w.scal + 24);
    }
    // Rayleigh-Ritz matrix T = Q^T W W^T Q: its eigenvectors order the basis (largest
    // energy first); the energies themselves are taken from the projections below.
    const long long RK = (long long)CM * K;
    if (kr) {
        // budget scale: the norm of the column-normalised weights,
        // sum_{k,j} (xa_k xb_j)^2 prod_l nu_l(k,j)^2 with nu_l(k,j)^2 = ((E_l.E_l)^T (Yh_l.Yh_l))[k,j]
        gemm_p(bp, st, kr->Ra, kr->S, n, LdSqT{kr->E, n, kr->bsE}, LdSqN{kr->Yh, n, (long long)n * h->KIN},
             1.0, 0.0, w.Nu, kr->Ra, (long long)std::max(h->RA, h->RP) * h->KIN, d);
        launch_inner_reduce(st, d, kr->Ra, kr->S, kr->xa, kr->xb, w.Nu, kr->Ra,
                            (long long)std::max(h->RA, h->RP) * h->KIN, w.scal + 4, true);
        // per mode, the weights that turn the columns e_lk . y_lj into those of the
        // column-normalised tensor (the energies below are measured with them)
        launch_kr_norm_weights(st, d, kr->Ra, kr->S, kr->xa, kr->xb, w.Nu, kr->Ra,
                               (long long)std::max(h->RA, h->RP) * h->KIN, w.wN, h->KMAX);
        launch_outer_weights(st, kr->Ra, kr->xa, kr->S, kr->xb, w.wK);
        // projections of every term onto the basis: B2t_l = Q_l^T (Et_l . Yh_l) (cs x rE S)
        // through the compressed symbol factors, then Cq_l[:, (k,j)] = sum_a B2t_l[:, (a,j)]
        // Mt_l[a,k] (one GEMM per mode, batched over the S input columns j)
        const long long RKt = (long long)CM * Kt;
        gemm_p(h->prec, st, cs, (int)Kt, n, LdT{Qb, n, nC},
             LdKR{kr->Et, n, kr->bsEt, kr->Yh, n, (long long)n * h->KIN, kr->S}, 1.0, 0.0, w.C2, CM,
             RKt, d);
        for (int l = 0; l < d; ++l)
            gemm_p(h->prec, st, cs, kr->Ra, kr->rE, LdColsJ{w.C2 + l * RKt, CM, kr->S},
                 LdN{kr->Mt + l * kr->bsMt, kr->rE, 0}, 1.0, 0.0, w.Cq + l * RK, CM * kr->S, CM,
                 kr->S);
        // T_l = Cq_l diag(w_l^2) Cq_l^T with the column-normalised weights of mode l
        gemm_p(h->prec, st, cs, cs, (int)K, LdSq{w.Cq, CM, RK, w.wN, h->KMAX}, LdT{w.Cq, CM, RK},
               1.0, 0.0, w.Tr, CM, CC, d);
    } else {
        // Bq = Q^T W (cs x K) in w.C, T = Bq Bq^T
        double* Bq = w.C;
        gemm_p(h->prec, st, cs, (int)K, n, LdT{Qb, n, nC}, LdAbsN{dn->U, dn->ld, dn->bs, dn->w}, 1.0, 0.0, Bq,
             CM, (long long)CM * K, d);
        gemm(st, cs, cs, (int)K, LdN{Bq, CM, (long long)CM * K}, LdT{Bq, CM, (long long)CM * K}, 1.0,
             0.0, w.Tr, CM, CC, d);
        launch_sumsq(st, (int)K, dn->w, w.scal + 4, 1);
    }
    CKL();
    // both Rayleigh-Ritz matrices come from projected rows (row-graded).  The energies that
    // decide the ranks are measured by projection for whatever basis the solver returns, so
    // off-diagonal entries far below the stage-1 budget (eps ||w||)^2 / (2d) need no rotation:
    // they are skipped below 1 % of it
    launch_gjacobi(st, d, w.Tr, CM, CC, dims + D_C1, 1, cs, w.theta, CM, w.Vr, CM, CC, false,
                   1e-20f, w.scal + 4, kEnergyFloor * eps * eps / (2.0 * d));
    // Zc_l = Q_l Vr_l (all cs Ritz directions, descending)
    gemm_p(bp, st, n, cs, cs, LdN{Qb, n, nC}, LdN{w.Vr, CM, CC}, 1.0, 0.0, w.Z, n, nC, d);
    // B2_l = Zc_l^T U_l (cs x K, unweighted): its first r_l rows are the projected factors C_l
    // of the core; rho_i = sum_K w_K^2 B2[i, K]^2 is the energy of W_l along Ritz direction i
    const double* wK = dn ? dn->w : w.wK;
    if (kr) {
        // C_l = Vr_l^T Cq_l: the projections of the terms onto the Ritz directions; the energy
        // of mode l's column-normalised side matrix along direction i is
        // sum_{(k,j)} w_l[k,j]^2 C_l[i,(k,j)]^2
        gemm_p(h->prec, st, cs, (int)K, cs, LdT{w.Vr, CM, CC}, LdN{w.Cq, CM, RK}, 1.0, 0.0, w.C,
               CM, RK, d);
        launch_row_energy(st, d, cs, (int)K, w.C, CM, RK, w.wN, w.theta, CM, h->KMAX);
    } else {
        gemm_p(h->prec, st, cs, (int)K, n, LdT{w.Z, n, nC}, LdN{dn->U, dn->ld, dn->bs}, 1.0, 0.0, w.C, CM, RK,
             d);
        launch_row_energy(st, d, cs, (int)K, w.C, CM, RK, wK, w.theta, CM);
    }
    // Tucker ranks: smallest r_l with sum_{i >= r_l} rho_i + missed <= (eps ||w||_2)^2 / (2d)
    launch_select_tucker(st, d, w.theta, CM, w.scal + 24, w.scal + 4, eps * eps / (2.0 * d),
                         std::min(RM, cs), dims + D_R, w.scal + 8, dims + D_C1);
    launch_stage2_dims(st, d, dims);
    const int rz = std::min(RM, cs);
    CKL();
    // ---- core: B3[(a + r0 b), c] = sum_K w_K C0[a,K] C1[b,K] C2[c,K] ----------------------
    const int RR = RM * RM;
    if (h->prec == GP_TC64) {
        // tensor-core form: the weights are folded into the mode-1 factor first (C1 is not
        // used after the core), so an operand element is a product of two factors, whose
        // digits are formed from the exact mantissa product
        launch_scale_cols(st, CM, (int)K, w.C + RK, CM, wK);
        LdCoreW A{w.C, w.C + RK, CM, dims + D_R};
        if (d == 3)
            gemm_p(h->prec, st, RR, RM, (int)K, A, LdT{w.C + 2 * RK, CM, 0}, 1.0, 0.0, w.core, RR, 0,
                   1, dims + D_R12, dims + D_R3, nullptr);
        else
            gemm_p(h->prec, st, RR, 1, (int)K, A, LdOnes{}, 1.0, 0.0, w.core, RR, 0, 1, dims + D_R12,
                   nullptr, nullptr);
    } else {
        LdCore A{w.C, w.C + RK, wK, CM, dims + D_R};
        if (d == 3)
            gemm_p(h->prec, st, RR, RM, (int)K, A, LdT{w.C + 2 * RK, CM, 0}, 1.0, 0.0, w.core, RR, 0,
                   1, dims + D_R12, dims + D_R3, nullptr);
        else
            gemm_p(h->prec, st, RR, 1, (int)K, A, LdOnes{}, 1.0, 0.0, w.core, RR, 0, 1, dims + D_R12,
                   nullptr, nullptr);
    }
    CKL();
    launch_core_energy(st, d, w.core, RR, dims, w.scal + 12);
    // mode-3 rotation: G3 = B3^T B3, W3 = eigvecs, Srot = B3 W3
    gemm(st, RM, RM, RR, LdT{w.core, RR, 0}, LdN{w.core, RR, 0}, 1.0, 0.0, w.G3, RM, 0, 1,
         dims + D_R3, dims + D_R3, dims + D_R12);
    // stage-2 Grams: the same floor against the stage-2 budget (eps ||core||)^2 / 2
    launch_gjacobi(st, 1, w.G3, RM, 0, dims + D_R3, 0, RM, w.ev3, 0, w.W3, RM, 0, false, 1e-20f,
                   w.scal + 12, kEnergyFloor * eps * eps / 2.0);
    gemm(st, RR, RM, RM, LdN{w.core, RR, 0}, LdN{w.W3, RM, 0}, 1.0, 0.0, w.Srot, RR, 0, 1,
         dims + D_R12, dims + D_R3, dims + D_R3);
    // slice Grams SG[s] = S_s^T S_s  (S_s = r0 x r1, compact column s of Srot)
    gemm(st, RM, RM, RM, LdSlT{w.Srot, RR, dims + D_R}, LdSl{w.Srot, RR, dims + D_R}, 1.0, 0.0,
         w.SG, RM, RR, (d == 3) ? RM : 1, dims + D_R + 1, dims + D_R + 1, dims + D_R);
    launch_gjacobi(st, (d == 3) ? RM : 1, w.SG, RM, RR, dims + D_R + 1, 0, RM, w.mus, RM, w.Vs, RM, RR, false,
                   1e-20f, w.scal + 12, kEnergyFloor * eps * eps / 2.0);
    // candidate term energies ||S_s y_i||^2 taken directly (not the Gram eigenvalues)
    launch_slice_energy(st, (d == 3) ? RM : 1, RM, dims, w.Srot, RR, w.Vs, RM, RR, w.mus, RM);
    CKL();
    launch_select_terms(st, w.mus, RM, dims + D_R3, dims + D_NPER, RM, RM, w.scal + 12,
                        eps * eps / 2.0, maxq, dims + D_Q, w.sigma, w.tslice, w.tidx, w.scal + 16);
    const long long RQ = (long long)RM * h->QMAX;
    launch_gather_terms(st, d, RM, dims, dims + D_Q, maxq, w.sigma, w.tslice, w.tidx, w.Srot, RR,
                        w.W3, RM, w.Vs, RM, RR, w.X, RM, RQ);
    CKL();
    // ---- output factors U'_l = Z_l X_l (eigen-index domain: F (Z_l X_l)) ------------------
    const double* Zuse = w.Z;
    if (kr && !h->spectral) {
        const double* in[3] = {w.Z, w.Z + nC, w.Z + 2 * nC};
        double* o[3] = {w.Zr, w.Zr + nC, w.Zr + 2 * nC};
        eig_transform_cols(h, st, rz, in, n, o, n, false);
        Zuse = w.Zr;
    }
    for (int l = 0; l < d; ++l)
        gemm_p(bp, st, n, maxq, RM, LdN{Zuse + l * nC, n, 0}, LdN{w.X + l * RQ, RM, 0}, 1.0, 0.0,
               out.U[l], out.ld, 0, 1, nullptr, dims + D_Q, dims + D_R + l);
    CK(cudaMemcpyAsync(out.xi, w.sigma, sizeof(double) * maxq, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->hint, dims, sizeof(int) * D_SIZE, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (int rc_ = tc_status(h)) return rc_;
    out.rank = h->hint[D_Q];
    for (int l = 0; l < d; ++l) {
        h->stat_rsum += h->hint[D_R + l];
        h->stat_rcount += 1;
        h->stat_rmax = std::max(h->stat_rmax, h->hint[D_R + l]);
        h->stat_bmax = std::max(h->stat_bmax, h->hint[D_C1 + l]);
    }
    return FC_OK;
}

// Khatri-Rao input from a CP tensor x and a symbol: Yh = F x (DST of the x factors)
// which: 0 = operator symbol, 1 = preconditioner, 2 = state symbol beta rho^-alpha
int kr_from(fc_ctx* h, cudaStream_t st, const CP& x, int which, KRIn& kr) {
    if (x.rank > h->KIN) return FC_ERANK;
    const long long nK = (long long)h->n * h->KIN;
    const double* in[3] = {x.U[0], x.U[1], x.U[2]};
    double* o[3] = {h->w.Yh, h->w.Yh + nK, h->w.Yh + 2 * nK};
    if (h->spectral) {                    // already in the eigenbasis: copy the factors
        for (int l = 0; l < h->d; ++l)
            if (x.rank > 0)
                CK(cudaMemcpy2DAsync(o[l], sizeof(double) * h->n, in[l], sizeof(double) * x.ld,
                                     sizeof(double) * h->n, x.rank, cudaMemcpyDeviceToDevice, st));
    } else {
        eig_transform_cols(h, st, x.rank, in, x.ld, o, h->n, true);
    }
    if (which == 1) {
        kr.xa = h->xiP; kr.E = h->EP; kr.Ra = h->RP; kr.bsE = (long long)h->n * h->RP;
    } else if (which == 2) {
        kr.xa = h->xiS; kr.E = h->EA; kr.Ra = h->RS; kr.bsE = (long long)h->n * h->RA;
    } else {
        kr.xa = h->xiA; kr.E = h->EA; kr.Ra = h->RA; kr.bsE = (long long)h->n * h->RA;
    }
    const int sidx = (which == 1) ? 1 : (which == 2 ? 2 : 0);
    kr.rE = h->rE[sidx];
    kr.Et = h->Et[sidx];
    kr.bsEt = (long long)h->n * kr.rE;
    kr.Mt = h->Mt[sidx];
    kr.bsMt = (long long)kr.rE * kr.Ra;
    kr.xb = x.xi;
    kr.Yh = h->w.Yh;
    kr.S = x.rank;
    // the E arrays use batch stride n * RA for both symbols (see fc_setup)
    return FC_OK;
}

int inner_impl(fc_ctx* h, cudaStream_t st, const CP& x, const CP& y, double* out) {
    if (x.rank == 0 || y.rank == 0) { *out = 0.0; return FC_OK; }
    if (x.rank > h->KIN || y.rank > h->KIN) return FC_ERANK;
    const long long kk = (long long)h->KIN * h->KIN;
    // the cross-Grams of the factors: tensor-core digits in form 3 (FP64-accurate), else FP64;
    // the recurrence itself (the weighted sum below and the scalars) is FP64 in every form
    const int bp = (h->prec == GP_TC64) ? GP_TC64 : GP_F64;
    for (int l = 0; l < h->d; ++l)
        gemm_p(bp, st, x.rank, y.rank, h->n, LdT{x.U[l], x.ld, 0}, LdN{y.U[l], y.ld, 0}, 1.0, 0.0,
               h->w.Mi + l * kk, x.rank);
    launch_inner_reduce(st, h->d, x.rank, y.rank, x.xi, y.xi, h->w.Mi, x.rank, kk, h->w.scal + 20);
    CKL();
    CK(cudaMemcpyAsync(h->hbuf, h->w.scal + 20, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = h->hbuf[0];
    return FC_OK;
}

// out = trunc(a*x + b*y) with column normalisation (CP linear combination of Algorithm 1)
int combo_trunc(fc_ctx* h, cudaStream_t st, const CP& x, double a, const CP* y, double b,
                double eps, int maxq, CP& out) {
    Piece p0{x.xi, {x.U[0], x.U[1], x.U[2]}, x.ld, x.rank, a};
    Piece p1{nullptr, {nullptr, nullptr, nullptr}, 0, 0, 0.0};
    if (y) p1 = Piece{y->xi, {y->U[0], y->U[1], y->U[2]}, y->ld, y->rank, b};
    const int K = p0.K + p1.K;
    if (K > h->w.cat.cap) return FC_ERANK;
    CP& cat = h->w.cat;
    launch_concat_normalize(st, h->d, h->n, p0, p1, cat.U[0], cat.ld, cat.bs(), cat.xi);
    CKL();
    cat.rank = K;
    DenseIn dn{cat.xi, cat.U[0], cat.ld, cat.bs(), K};
    return truncate_impl(h, st, nullptr, &dn, eps, maxq, out);
}

int kr_trunc(fc_ctx* h, cudaStream_t st, const CP& x, int which, double eps, int maxq, CP& out) {
    KRIn kr;
    int rc = kr_from(h, st, x, which, kr);
    if (rc) return rc;
    return truncate_impl(h, st, &kr, nullptr, eps, maxq, out);
}

}  // namespace

// =========================================================================================
extern "C" {

const char* fc_strerror(int code) {
    switch (code) {
        case FC_OK: return "ok";
        case FC_EINVAL: return "invalid argument";
        case FC_ERANK: return "rank capacity exceeded";
        case FC_ENOCONV: return "PCG did not converge within kmax iterations";
        case FC_EBREAKDOWN: return "PCG breakdown: <P, S> <= 0 after truncation";
        case FC_ENAN: return "non-finite PCG scalar";
        case FC_ECUDA: return "CUDA error";
        case FC_EWORKSPACE: return "workspace missing or too small";
        case FC_ESETUP: return "quadrature or preconditioner construction failed";
        case FC_ETIMEOUT: return "a bounded wait inside a kernel expired (tensor-core pipeline)";
        default: return "unknown error";
    }
}

const char* fc_last_cuda_error(void) { return g_cuda_msg.c_str(); }

int fc_symeig(int method, int batch, int m, const double* dev_A, int lda, long long strideA,
              double* dev_w, long long strideW, double* dev_V, int ldv, long long strideV,
              void* stream) {
    if (!(method == 0 || method == 1) || batch < 0 || m < 0 || m > kMaxC ||
        (batch > 0 && m > 0 && (!dev_A || !dev_w || !dev_V)) || lda < m || ldv < m)
        return FC_EINVAL;
    if (batch == 0 || m == 0) return FC_OK;
    if (int rc = ensure_attributes()) return rc;
    if (method == 0)
        launch_symeig((cudaStream_t)stream, batch, dev_A, lda, strideA, nullptr, 0, m, dev_w,
                      strideW, dev_V, ldv, strideV);
    else
        launch_gjacobi((cudaStream_t)stream, batch, dev_A, lda, strideA, nullptr, 0, m, dev_w,
                       strideW, dev_V, ldv, strideV, true);
    CKL();
    return FC_OK;
}

int fc_dgemm(int precision, int transA, int transB, int M, int N, int K, double alpha,
             const double* dev_A, int lda, const double* dev_B, int ldb, double beta,
             double* dev_C, int ldc, void* stream) {
    if (!(precision >= 0 && precision <= 2) || M < 0 || N < 0 || K < 0) return FC_EINVAL;
    if (M == 0 || N == 0) return FC_OK;
    if (!dev_C || ldc < M || (K > 0 && (!dev_A || !dev_B))) return FC_EINVAL;
    if (lda < (transA ? K : M) || ldb < (transB ? N : K) || lda < 1 || ldb < 1) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    auto run = [&](auto la, auto lb) -> int {
        if (precision == 2) {
            if (!gemm_tc(st, M, N, K, la, lb, alpha, beta, dev_C, ldc, 0, 1, nullptr, nullptr,
                         nullptr))
                return FC_ECUDA;
            CKL();
            CK(cudaStreamSynchronize(st));
            int flag = 0;
            CK(cudaMemcpyFromSymbol(&flag, g_tc_error, sizeof(int)));
            if (flag) {
                const int zero = 0;
                CK(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int)));
                return FC_ETIMEOUT;
            }
            return FC_OK;
        }
        gemm_p(precision == 1 ? GP_DF32 : GP_F64, st, M, N, K, la, lb, alpha, beta, dev_C, ldc);
        CKL();
        return FC_OK;
    };
    if (!transA && !transB) return run(LdN{dev_A, lda, 0}, LdN{dev_B, ldb, 0});
    if (!transA && transB) return run(LdN{dev_A, lda, 0}, LdT{dev_B, ldb, 0});
    if (transA && !transB) return run(LdT{dev_A, lda, 0}, LdN{dev_B, ldb, 0});
    return run(LdT{dev_A, lda, 0}, LdT{dev_B, ldb, 0});
}

int fc_prof_enable(int kclass) {
    if (kclass < 0 || kclass > KC_F64) return FC_EINVAL;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError());
    g_prof_used = 0;
    unsigned long long* w = prof_work_counter();
    if (!w) return FC_ECUDA;
    CK(cudaMemset(w, 0, sizeof(unsigned long long)));
    CK(cudaDeviceSynchronize());
    g_prof_class.store(kclass);
    return FC_OK;
}

int fc_prof_read(long long* launches, double* total_ms, double* work) {
    if (!launches || !total_ms || !work) return FC_EINVAL;
    g_prof_class.store(KC_NONE);
    std::lock_guard<std::mutex> lock(g_prof_mu);
    CK(cudaDeviceSynchronize());
    double tot = 0.0;
    for (size_t i = 0; i < g_prof_used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g_prof_events[i].first, g_prof_events[i].second));
        tot += ms;
    }
    unsigned long long wk = 0;
    unsigned long long* w = prof_work_counter();
    if (!w) return FC_ECUDA;
    CK(cudaMemcpy(&wk, w, sizeof(wk), cudaMemcpyDeviceToHost));
    *launches = (long long)g_prof_used;
    *total_ms = tot;
    *work = (double)wk;
    return FC_OK;
}

int fc_set_wait_limit(int iterations, int* previous) {
    if (iterations < 0) return FC_EINVAL;
    const int old = g_tc_wait_limit.exchange(iterations);
    if (previous) *previous = old;
    return FC_OK;
}

unsigned long long fc_launch_count(void) { return fc::g_launches.load(std::memory_order_relaxed); }

int fc_setup(int n, int d, double alpha, double beta, double gamma, double eps,
             const fc_setup_opts* o, fc_handle* out) {
    if (!out) return FC_EINVAL;
    *out = nullptr;
    if (!(d == 2 || d == 3) || n < 1 || n > 8191 || !(alpha > 0.0 && alpha <= 1.0) ||
        !(beta > 0.0) || !(gamma > 0.0) || !(eps > 0.0) || !std::isfinite(beta) ||
        !std::isfinite(gamma))
        return FC_EINVAL;
    fc_setup_opts opts{1e-10, 24, 32, 48, 0, 0, 0, 0, 0};
    if (o) {
        if (!(o->op_kind >= 0 && o->op_kind <= 2) || !(o->precond_kind == 0 || o->precond_kind == 1))
            return FC_EINVAL;
        opts.op_kind = o->op_kind;
        opts.precond_kind = o->precond_kind;
        opts.directional = o->directional ? 1 : 0;
        opts.precision = (o->precision == 1 || o->precision == 2) ? o->precision : 0;
        if (o->delta_sym > 0) opts.delta_sym = o->delta_sym;
        if (o->precond_rank > 0) opts.precond_rank = o->precond_rank;
        if (o->max_rank > 0) opts.max_rank = o->max_rank;
        if (o->max_tucker > 0) opts.max_tucker = o->max_tucker;
        if (o->max_input_rank > 0) opts.max_input_rank = o->max_input_rank;
    }
    opts.max_tucker = std::min(opts.max_tucker, kMaxC - 8);
    opts.max_rank = std::min(opts.max_rank, opts.max_tucker * opts.max_tucker);
    if (opts.max_input_rank <= 0) opts.max_input_rank = opts.max_rank;
    if (int rc_ = ensure_attributes()) return rc_;
    // Directionally fractional operator sum_l (-Delta_l)^alpha (Remark after Lemma 4.1): the
    // same eigenbasis with eigenvalues sum_l lambda^alpha, i.e. spectrum lambda^alpha and
    // exponent 1 in g = beta^2 rho^-1 + gamma rho.
    // Per-mode spectra: the closed-form DST-I eigenvalues, or for a mode with a coefficient
    // a_l (Remark on variable coefficients) the eigen-decomposition of its 1D stiffness matrix
    // of -(a_l u')', whose orthonormal eigenvectors replace the DST-I of that mode.
    bool varcoef = false;
    if (o)
        for (int l = 0; l < d; ++l) varcoef |= (o->coeff[l] != nullptr);
    std::vector<double> lam((size_t)3 * n, 0.0), Vh;
    if (varcoef) Vh.assign((size_t)3 * n * n, 0.0);
    {
        const std::vector<double> lam0 = spectrum(n);
        const double N1 = n + 1.0, sc = std::sqrt(2.0 / N1);
        for (int l = 0; l < d; ++l) {
            if (varcoef && o->coeff[l]) {
                for (int i = 0; i <= n; ++i)
                    if (!(o->coeff[l][i] > 0.0) || !std::isfinite(o->coeff[l][i])) return FC_EINVAL;
                std::vector<double> dg, off, lv, Vl;
                stiffness_1d(n, o->coeff[l], dg, off);
                if (!tridiag_eig(n, dg, off, lv, Vl)) return FC_ESETUP;
                std::copy(lv.begin(), lv.end(), lam.begin() + (size_t)l * n);
                std::copy(Vl.begin(), Vl.end(), Vh.begin() + (size_t)l * n * n);
            } else {
                std::copy(lam0.begin(), lam0.end(), lam.begin() + (size_t)l * n);
                if (varcoef)                       // this mode keeps the DST-I, stored explicitly
                    for (int k = 0; k < n; ++k)
                        for (int i = 0; i < n; ++i)
                            Vh[(size_t)l * n * n + i + (size_t)k * n] =
                                sc * std::sin(M_PI * (i + 1.0) * (k + 1.0) / N1);
            }
        }
    }
    double alpha_eff = alpha;
    if (opts.directional) {
        for (double& x : lam) x = std::pow(x, alpha);
        alpha_eff = 1.0;
    }
    double rmin = 0.0, rmax = 0.0;               // range of rho = sum_l lambda_{i_l, l}
    for (int l = 0; l < d; ++l) {
        rmin += lam[(size_t)l * n];
        rmax += lam[(size_t)l * n + n - 1];
    }
    // operator symbol: the control operator, or a test operator of Section 6
    SymbolSpec gs;
    if (opts.op_kind == 0) {
        gs.a = beta * beta; gs.sn = alpha_eff; gs.b = gamma; gs.sp = alpha_eff;
    } else if (opts.op_kind == 1) {                 // A^alpha
        gs.b = 1.0; gs.sp = alpha_eff;
    } else {                                        // I + A^(2 alpha), 2 alpha <= 1
        if (2.0 * alpha_eff > 1.0) return FC_EINVAL;
        gs.b = 1.0; gs.sp = 2.0 * alpha_eff; gs.c = 1.0;
    }
    SymbolNodes sym, pc;
    if (!build_symbol_nodes(rmin, rmax, d, gs, opts.delta_sym, sym)) return FC_ESETUP;
    if (opts.precond_kind == 1) {
        if (!build_inverse_power_nodes(rmin, rmax, d, alpha_eff, opts.delta_sym, pc)) return FC_ESETUP;
    } else if (!build_precond_nodes(rmin, rmax, gs, opts.precond_rank, pc)) {
        return FC_ESETUP;
    }
    fc_ctx* h = new (std::nothrow) fc_ctx();
    if (!h) return FC_EINVAL;
    h->n = n; h->d = d; h->alpha = alpha; h->beta = beta; h->gamma = gamma; h->eps = eps;
    h->alpha_eff = alpha_eff;
    h->spec = gs;
    h->prec = (opts.precision == 2) ? GP_TC64 : (opts.precision == 1) ? GP_DF32 : GP_F64;
    h->opts = opts;
    h->RA = (int)sym.tau.size();
    h->RS = sym.r_minus;
    h->RP = (int)pc.tau.size();
    h->CAP = opts.max_rank;
    h->KIN = std::max(opts.max_input_rank, opts.max_rank);
    h->RM = opts.max_tucker;
    h->QMAX = std::max(h->CAP, h->KIN);
    h->KMAX = std::max<long long>({(long long)h->RA * h->KIN, (long long)h->RP * h->KIN,
                                   2LL * h->CAP, (long long)h->KIN});
    // device tables
    const int N = n + 1;
    const int RAm = std::max(h->RA, h->RP);
    const bool pow2 = (N & (N - 1)) == 0 && N >= 2 && N <= 4096;
    size_t tcount = 3 * (size_t)n + 2 * N + 4 * ((size_t)h->RA + h->RP + h->RS) + 2 * 3 * (size_t)n * RAm +
                    (pow2 ? 2 * (size_t)N + 1 : 0) +
                    (varcoef ? 3 * (size_t)n * n : 0);
    if (cudaMalloc(&h->tables, tcount * sizeof(double)) != cudaSuccess) {
        delete h;
        return FC_ECUDA;
    }
    double* p = h->tables;
    h->lam = p; p += 3 * (size_t)n;
    h->sintab = p; p += 2 * N;
    if (varcoef) { h->V = p; p += 3 * (size_t)n * n; }
    h->xiA = p; p += h->RA;
    h->xiP = p; p += h->RP;
    h->EA = p; p += 3 * (size_t)n * RAm;
    h->EP = p; p += 3 * (size_t)n * RAm;

    h->xiS = p; p += h->RS;
    if (pow2) {                       // double2 table: 16-byte aligned start
        p = h->tables + (((size_t)(p - h->tables) + 1) & ~(size_t)1);
        h->twid = reinterpret_cast<double2*>(p);
        p += 2 * (size_t)N;
    }
    h->xiAw = p; p += 3 * (size_t)h->RA;
    h->xiPw = p; p += 3 * (size_t)h->RP;
    h->xiSw = p; p += 3 * (size_t)h->RS;
    std::vector<double> tab(2 * N);
    const double sc = std::sqrt(2.0 / N);
    for (int m = 0; m < 2 * N; ++m) {
        // sin(pi m / N) with the argument reduced into [0, pi/2] for accuracy
        int mm = m % (2 * N);
        double sgn = 1.0;
        if (mm >= N) { mm -= N; sgn = -1.0; }
        if (2 * mm > N) mm = N - mm;
        tab[m] = sc * sgn * std::sin(M_PI * mm / N);
    }
    cudaStream_t st = 0;
    int rc = FC_OK;
    int *dmode = nullptr;
    double *dtau = nullptr, *dw = nullptr;
    const int RT = h->RA + h->RP;
    std::vector<double> tau(RT), wv(RT);
    std::vector<int> mode(RT);
    for (int k = 0; k < h->RA; ++k) { tau[k] = sym.tau[k]; wv[k] = sym.w[k]; mode[k] = sym.mode[k]; }
    for (int k = 0; k < h->RP; ++k) { tau[h->RA + k] = pc.tau[k]; wv[h->RA + k] = pc.w[k]; mode[h->RA + k] = -1; }
    do {
        if ((varcoef && cudaMemcpy(h->V, Vh.data(), sizeof(double) * Vh.size(), cudaMemcpyHostToDevice)) ||
            cudaMemcpy(h->lam, lam.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice) ||
            cudaMemcpy(h->sintab, tab.data(), sizeof(double) * 2 * N, cudaMemcpyHostToDevice)) { rc = FC_ECUDA; break; }
        if (pow2) {
            // e^{-i pi k / N}: angle reduced to [0, pi/2] by the symmetries of sin and cos
            std::vector<double> tw(2 * (size_t)N);
            for (int k = 0; k < N; ++k) {
                int q = k;
                double c, sn_;
                if (2 * q <= N) { c = std::cos(M_PI * q / N); sn_ = std::sin(M_PI * q / N); }
                else { q = N - k; c = -std::cos(M_PI * q / N); sn_ = std::sin(M_PI * q / N); }
                tw[2 * (size_t)k] = c;
                tw[2 * (size_t)k + 1] = -sn_;
            }
            if (cudaMemcpy(h->twid, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice)) {
                rc = FC_ECUDA; break;
            }
        }
        if (cudaMalloc(&dtau, sizeof(double) * RT) || cudaMalloc(&dw, sizeof(double) * RT) ||
            cudaMalloc(&dmode, sizeof(int) * RT)) { rc = FC_ECUDA; break; }
        cudaMemcpy(dtau, tau.data(), sizeof(double) * RT, cudaMemcpyHostToDevice);
        cudaMemcpy(dw, wv.data(), sizeof(double) * RT, cudaMemcpyHostToDevice);
        cudaMemcpy(dmode, mode.data(), sizeof(int) * RT, cudaMemcpyHostToDevice);
        const long long bsE = (long long)n * h->RA;
        const long long bsP = (long long)n * h->RP;
        launch_build_symbol(st, n, d, h->lam, n, dtau, dw, dmode, h->RA, h->EA, n, bsE, h->xiA);
        launch_build_symbol(st, n, d, h->lam, n, dtau + h->RA, dw + h->RA, dmode + h->RA, h->RP, h->EP,
                            n, bsP, h->xiP);
        // state symbol beta rho^-alpha = (beta^2 rho^-alpha part of the control symbol) / beta
        launch_copy_weights(st, h->RS, h->xiA, 1.0 / beta, h->xiS);
        if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = FC_ECUDA; break; }
        if ((rc = symbol_proxy_weights(h)) != FC_OK) break;
    } while (0);
    cudaFree(dtau); cudaFree(dw); cudaFree(dmode);
    if (rc == FC_OK) rc = compress_symbols(h);
    if (rc == FC_OK && (cudaMallocHost(&h->hbuf, 64 * sizeof(double)) != cudaSuccess ||
                        cudaMallocHost(&h->hint, 64 * sizeof(int)) != cudaSuccess))
        rc = FC_ECUDA;
    if (rc != FC_OK) {
        fc_destroy(h);
        return rc;
    }
    // precond symbol's E uses mode stride n*RP; KRIn uses n*RA for E: store a view note
    fc_setup_info& I = h->info;
    I.n = n; I.d = d;
    I.rank_symbol = h->RA; I.rank_minus = sym.r_minus; I.rank_plus = sym.r_plus;
    I.rank_precond = h->RP;
    I.rho_min = sym.rho_min; I.rho_max = sym.rho_max;
    I.sym_err = sym.err; I.pc_err = pc.err;
    Arena a;
    I.workspace_bytes = layout(h, a);
    *out = h;
    return FC_OK;
}

int fc_get_info(fc_handle h, fc_setup_info* info) {
    if (!h || !info) return FC_EINVAL;
    *info = h->info;
    return FC_OK;
}

int fc_workspace_size(fc_handle h, size_t* bytes) {
    if (!h || !bytes) return FC_EINVAL;
    *bytes = h->info.workspace_bytes;
    return FC_OK;
}

int fc_set_workspace(fc_handle h, void* dev_ptr, size_t bytes) {
    if (!h || !dev_ptr || bytes < h->info.workspace_bytes) return FC_EWORKSPACE;
    if (((uintptr_t)dev_ptr & 255) != 0) return FC_EINVAL;
    Arena a;
    a.base = (char*)dev_ptr;
    a.cap = bytes;
    a.count_only = false;
    layout(h, a);
    h->ws = (char*)dev_ptr;
    h->ws_bytes = bytes;
    return FC_OK;
}

int fc_get_symbol(fc_handle h, int which, fc_cp* out, void* stream) {
    if (!h || !out || !(which >= 0 && which <= 2) || !check_cp(h, out, true)) return FC_EINVAL;
    const int R = which == 1 ? h->RP : (which == 2 ? h->RS : h->RA);
    if (out->cap < R) { out->rank = R; return FC_ERANK; }
    cudaStream_t st = (cudaStream_t)stream;
    const double* xi = which == 1 ? h->xiP : (which == 2 ? h->xiS : h->xiA);
    const double* E = which == 1 ? h->EP : h->EA;
    const long long bs = (long long)h->n * (which == 1 ? h->RP : h->RA);
    CK(cudaMemcpyAsync(out->xi, xi, sizeof(double) * R, cudaMemcpyDeviceToDevice, st));
    for (int l = 0; l < h->d; ++l)
        CK(cudaMemcpy2DAsync(out->U[l], sizeof(double) * out->ld, E + l * bs, sizeof(double) * h->n,
                             sizeof(double) * h->n, R, cudaMemcpyDeviceToDevice, st));
    out->rank = R;
    CK(cudaStreamSynchronize(st));
    return FC_OK;
}

static int apply_common(fc_handle h, const fc_cp* x, fc_cp* y, void* stream, bool precond) {
    if (!h || !check_cp(h, x, false) || !check_cp(h, y, true)) return FC_EINVAL;
    if (!h->ws) return FC_EWORKSPACE;
    const int R = precond ? h->RP : h->RA;
    const long long K = (long long)R * x->rank;
    if (K > y->cap) { y->rank = (int)std::min<long long>(K, 0x7fffffff); return FC_ERANK; }
    cudaStream_t st = (cudaStream_t)stream;
    HandleCall call(h, st);
    if (call.rc) return call.rc;
    CP xc = from_user(x);
    KRIn kr;
    int rc = kr_from(h, st, xc, precond ? 1 : 0, kr);
    if (rc) return rc;
    // y_l = F (E_l[:,k] . Yh_l[:,j]) for all (k, j), weights xa_k xb_j (F: the inverse
    // transform of mode l, DST-I or the stiffness eigenbasis V_l)
    LdSine F{h->sintab, 2 * (h->n + 1)};
    const long long bsE = (long long)h->n * R;
    for (int l = 0; l < h->d; ++l) {
        const LdKR kl{kr.E + l * bsE, h->n, 0, kr.Yh + (long long)l * h->n * h->KIN, h->n, 0, kr.S};
        if (h->V)
            gemm_p(h->prec, st, h->n, (int)K, h->n, LdN{h->V + (long long)l * h->n * h->n, h->n, 0},
                   kl, 1.0, 0.0, y->U[l], y->ld);
        else
            gemm_p(h->prec, st, h->n, (int)K, h->n, F, kl, 1.0, 0.0, y->U[l], y->ld);
    }
    launch_outer_weights(st, R, kr.xa, kr.S, kr.xb, y->xi);
    CKL();
    y->rank = (int)K;
    if ((rc = flag_to_host(h, st))) return rc;
    CK(cudaStreamSynchronize(st));
    return tc_status(h);
}

int fc_apply(fc_handle h, const fc_cp* x, fc_cp* y, void* stream) {
    return apply_common(h, x, y, stream, false);
}
int fc_precond(fc_handle h, const fc_cp* x, fc_cp* y, void* stream) {
    return apply_common(h, x, y, stream, true);
}

int fc_truncate(fc_handle h, const fc_cp* x, double eps, int max_rank, int normalize, fc_cp* y,
                void* stream) {
    if (!h || !check_cp(h, x, false) || !check_cp(h, y, true) || !(eps >= 0.0) || max_rank < 1)
        return FC_EINVAL;
    if (!h->ws) return FC_EWORKSPACE;
    if (x->rank > h->w.cat.cap || x->rank > h->KMAX) { y->rank = x->rank; return FC_ERANK; }
    cudaStream_t st = (cudaStream_t)stream;
    HandleCall call(h, st);
    if (call.rc) return call.rc;
    CP xc = from_user(x), yc = from_user(y);
    int rc;
    if (normalize) {
        rc = combo_trunc(h, st, xc, 1.0, nullptr, 0.0, eps, max_rank, yc);
    } else {
        // copy into the contiguous concat buffer as given (no normalisation)
        CP& cat = h->w.cat;
        for (int l = 0; l < h->d; ++l)
            CK(cudaMemcpy2DAsync(cat.U[l], sizeof(double) * cat.ld, x->U[l], sizeof(double) * x->ld,
                                 sizeof(double) * h->n, x->rank, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(cat.xi, x->xi, sizeof(double) * x->rank, cudaMemcpyDeviceToDevice, st));
        DenseIn dn{cat.xi, cat.U[0], cat.ld, cat.bs(), x->rank};
        rc = truncate_impl(h, st, nullptr, &dn, eps, max_rank, yc);
    }
    y->rank = yc.rank;
    return rc;
}

int fc_state(fc_handle h, const fc_cp* u, double eps, int max_rank, fc_cp* y, void* stream) {
    if (!h || h->RS == 0) return FC_EINVAL;   // only the control operator has a state symbol
    return fc_apply_trunc(h, 2, u, eps, max_rank, y, stream);
}

int fc_apply_trunc(fc_handle h, int which, const fc_cp* x, double eps, int max_rank, fc_cp* y,
                   void* stream) {
    if (!h || !(which >= 0 && which <= 2) || (which == 2 && h->RS == 0) || !check_cp(h, x, false) || !check_cp(h, y, true) ||
        !(eps >= 0.0) || max_rank < 1)
        return FC_EINVAL;
    if (!h->ws) return FC_EWORKSPACE;
    if (x->rank > h->KIN) { y->rank = x->rank; return FC_ERANK; }
    HandleCall call(h, (cudaStream_t)stream);
    if (call.rc) return call.rc;
    CP xc = from_user(x), yc = from_user(y);
    int rc = kr_trunc(h, (cudaStream_t)stream, xc, which, eps, max_rank, yc);
    y->rank = yc.rank;
    return rc;
}

int fc_inner(fc_handle h, const fc_cp* x, const fc_cp* y, double* out_host, void* stream) {
    if (!h || !out_host || !check_cp(h, x, false) || !check_cp(h, y, false)) return FC_EINVAL;
    if (!h->ws) return FC_EWORKSPACE;
    return inner_impl(h, (cudaStream_t)stream, from_user(x), from_user(y), out_host);
}

int fc_solve(fc_handle h, const fc_cp* rhs, fc_cp* u, const fc_solve_opts* o,
             fc_solve_info* info, void* stream) {
    if (!h || !check_cp(h, rhs, false) || !check_cp(h, u, true)) return FC_EINVAL;
    if (!h->ws) return FC_EWORKSPACE;
    fc_solve_opts opts{1e-8, 0.0, 100, 0, 0, 0, 0};
    if (o) opts = *o;
    if (!(opts.tol > 0.0)) opts.tol = 1e-8;
    if (opts.kmax <= 0) opts.kmax = 100;
    if (opts.precision < 0 || opts.precision > 3 || opts.stall < 0) return FC_EINVAL;
    const double eps = (opts.eps > 0.0) ? opts.eps : h->eps;
    const int cap = std::min(h->CAP, (opts.max_rank > 0) ? opts.max_rank : h->CAP);
    if (u->cap < cap) { u->rank = cap; return FC_ERANK; }
    if (rhs->rank > h->KIN) return FC_ERANK;
    fc_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    h->stat_rsum = h->stat_rcount = 0;
    h->stat_rmax = h->stat_bmax = 0;
    h->seed = fc_ctx::kSeed0;  // same sketches for every solve of a right-hand side: reproducible
    cudaStream_t st = (cudaStream_t)stream;
    // contraction form of this solve: the handle's, or opts.precision - 1
    HandleCall call(h, st, opts.precision > 0 ? (opts.precision == 3 ? GP_TC64 :
                                                 opts.precision == 2 ? GP_DF32 : GP_F64) : -1);
    if (call.rc) return call.rc;
    auto& w = h->w;
    CP B = from_user(rhs);
    CP &X = w.Xs, &R = w.Rs, &P = w.Ps, &Z = w.Zs, &S = w.Ss, &Xb = w.Xb;
    int rc;
    double bn2;
    if ((rc = inner_impl(h, st, B, B, &bn2))) return rc;
    X.rank = 0;
    Xb.rank = 0;
    double bscale = 1.0;
    // the iterate returned: X, or with stall detection on an unconverged exit the iterate of
    // the smallest residual (Xb)
    bool use_best = false;
    auto finish = [&](int status) -> int {
        const CP& Xr = use_best ? Xb : X;
        inf.status = status;
        inf.rank_x = Xr.rank;
        inf.tucker_max = h->stat_rmax;
        inf.basis_max = h->stat_bmax;
        inf.tucker_mean = h->stat_rcount ? (double)h->stat_rsum / h->stat_rcount : 0.0;
        // X to the caller's u (spectral-resident: transformed back from the eigenbasis)
        if (h->spectral && Xr.rank > 0) {
            const double* xin[3] = {Xr.U[0], Xr.U[1], Xr.U[2]};
            double* uo[3] = {u->U[0], u->U[1], u->U[2]};
            eig_transform_cols(h, st, Xr.rank, xin, Xr.ld, uo, u->ld, false);
        } else {
            for (int l = 0; l < h->d; ++l)
                if (Xr.rank > 0)
                    CK(cudaMemcpy2DAsync(u->U[l], sizeof(double) * u->ld, Xr.U[l], sizeof(double) * Xr.ld,
                                         sizeof(double) * h->n, Xr.rank, cudaMemcpyDeviceToDevice, st));
        }
        if (Xr.rank > 0) launch_copy_weights(st, Xr.rank, Xr.xi, bscale, u->xi);   // undo 1/||B||
        u->rank = Xr.rank;
        if (int rf = flag_to_host(h, st)) return rf;
        CK(cudaStreamSynchronize(st));
        if (status == FC_OK && tc_status(h)) status = FC_ETIMEOUT;
        inf.status = status;
        if (info) *info = inf;
        return status;
    };
    if (!(bn2 > 0.0)) return finish(std::isfinite(bn2) ? FC_OK : FC_ENAN);
    const double bn = std::sqrt(bn2);
    // The iteration runs on B / ||B|| (all iterates O(1); the truncation thresholds and the
    // stopping test are relative, so this only fixes the scale); X is scaled back at exit.
    bscale = bn;
    // R0 = B / ||B|| (normalised columns, same tensor), X0 = 0
    {
        Piece p0{B.xi, {B.U[0], B.U[1], B.U[2]}, B.ld, B.rank, 1.0 / bn};
        Piece p1{nullptr, {nullptr, nullptr, nullptr}, 0, 0, 0.0};
        launch_concat_normalize(st, h->d, h->n, p0, p1, R.U[0], R.ld, R.bs(), R.xi);
        CKL();
        R.rank = B.rank;
        if (opts.spectral && R.rank > 0) {
            // spectral-resident iteration: R0 in the eigenbasis (unit columns stay unit)
            const long long nK = (long long)h->n * h->KIN;
            const double* rin[3] = {R.U[0], R.U[1], R.U[2]};
            double* tmp[3] = {w.Yh, w.Yh + nK, w.Yh + 2 * nK};
            eig_transform_cols(h, st, R.rank, rin, R.ld, tmp, h->n, true);
            for (int l = 0; l < h->d; ++l)
                CK(cudaMemcpy2DAsync(R.U[l], sizeof(double) * R.ld, tmp[l], sizeof(double) * h->n,
                                     sizeof(double) * h->n, R.rank, cudaMemcpyDeviceToDevice, st));
        }
    }
    h->spectral = opts.spectral != 0;
    struct SpectralReset {
        fc_ctx* h;
        ~SpectralReset() { h->spectral = false; }
    } spectral_reset{h};
    auto track = [&](const CP& c) { inf.max_rank_seen = std::max(inf.max_rank_seen, c.rank); ++inf.trunc_calls; };
    if ((rc = kr_trunc(h, st, R, 1, eps, cap, Z))) return rc;           // Z0 = trunc(precond(R0))
    track(Z);
    // P0 = Z0
    for (int l = 0; l < h->d; ++l)
        CK(cudaMemcpyAsync(P.U[l], Z.U[l], sizeof(double) * h->n * Z.rank, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(P.xi, Z.xi, sizeof(double) * Z.rank, cudaMemcpyDeviceToDevice, st));
    P.rank = Z.rank;
    double rz;
    if ((rc = inner_impl(h, st, R, Z, &rz))) return rc;
    // stall detection (opts.stall > 0): the run ends once `stall` iterations in a row have not
    // brought the recursive residual 10% below the last value that did
    double best = INFINITY, anchor = INFINITY;
    int since = 0;
    for (int k = 0; k < opts.kmax; ++k) {
        if ((rc = kr_trunc(h, st, P, 0, eps, cap, S))) return rc;        // S = trunc(fun(P))
        track(S);
        double ps;
        if ((rc = inner_impl(h, st, P, S, &ps))) return rc;
        if (!std::isfinite(ps) || !std::isfinite(rz)) { inf.iters = k; return finish(FC_ENAN); }
        if (!(ps > 0.0)) { inf.iters = k; return finish(FC_EBREAKDOWN); }
        const double a = rz / ps;                                             // alpha_k
        if (X.rank == 0) {
            if ((rc = combo_trunc(h, st, P, a, nullptr, 0.0, eps, cap, X))) return rc;
        } else {
            if ((rc = combo_trunc(h, st, X, 1.0, &P, a, eps, cap, X))) return rc;  // X + alpha P
        }
        track(X);
        if ((rc = combo_trunc(h, st, R, 1.0, &S, -a, eps, cap, R))) return rc;     // R - alpha S
        track(R);
        double rr;
        if ((rc = inner_impl(h, st, R, R, &rr))) return rc;
        const double rel = std::sqrt(std::max(rr, 0.0));          // ||R|| / ||B||
        if (k < 128) inf.history[k] = rel;
        inf.iters = k + 1;
        inf.relres = rel;
        if (!std::isfinite(rel)) return finish(FC_ENAN);
        if (rel <= opts.tol) return finish(FC_OK);
        if (opts.stall > 0) {
            if (rel < best) {                                   // keep the best iterate
                best = rel;
                for (int l = 0; l < h->d; ++l)
                    CK(cudaMemcpyAsync(Xb.U[l], X.U[l], sizeof(double) * h->n * X.rank,
                                       cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(Xb.xi, X.xi, sizeof(double) * X.rank, cudaMemcpyDeviceToDevice, st));
                Xb.rank = X.rank;
            }
            if (rel <= 0.9 * anchor) { anchor = rel; since = 0; }
            else if (++since >= opts.stall) { use_best = true; inf.relres = best; return finish(FC_ENOCONV); }
        }
        if ((rc = kr_trunc(h, st, R, 1, eps, cap, Z))) return rc;          // Z = trunc(precond(R))
        track(Z);
        double rzn;
        if ((rc = inner_impl(h, st, R, Z, &rzn))) return rc;
        const double b = rzn / rz;                                            // beta_k
        if ((rc = combo_trunc(h, st, Z, 1.0, &P, b, eps, cap, P))) return rc;  // P = Z + beta P
        track(P);
        rz = rzn;
    }
    if (opts.stall > 0 && Xb.rank > 0) { use_best = true; inf.relres = best; }
    return finish(FC_ENOCONV);
}

// Host threads of fc_solve_batched: at most kMaxWorkers (the schedule's `workers`, 16 unless
// set or tuned: enough to keep the GPU busy with latency-bound solves, few enough not to
// oversubscribe the host's cores).
constexpr int kMaxWorkers = 64;

namespace {
// Non-blocking streams of the batch workers per device, created on first use and kept for
// the life of the process (a solve is a chain of small launches and host synchronisations on
// its worker's stream).
struct WorkerStreams {
    std::mutex mu;
    cudaStream_t s[64][kMaxWorkers] = {};
    int made[64] = {};
};
WorkerStreams g_workers;

int worker_streams(int dev, int count, cudaStream_t* out) {
    if (dev < 0 || dev >= 64 || count < 1 || count > kMaxWorkers) return FC_EINVAL;
    std::lock_guard<std::mutex> lock(g_workers.mu);
    for (; g_workers.made[dev] < count; ++g_workers.made[dev])
        CK(cudaStreamCreateWithFlags(&g_workers.s[dev][g_workers.made[dev]], cudaStreamNonBlocking));
    for (int i = 0; i < count; ++i) out[i] = g_workers.s[dev][i];
    return FC_OK;
}
}  // namespace

int fc_get_schedule(fc_schedule* out) {
    if (!out) return FC_EINVAL;
    out->gemm_cover = sched(g_sched.gemm_cover);
    out->gemm_split = sched(g_sched.gemm_split);
    out->tc_split = sched(g_sched.tc_split);
    out->tc_min_log2 = sched(g_sched.tc_min_log2);
    out->workers = sched(g_sched.workers);
    out->order = sched(g_sched.order);
    return FC_OK;
}

int fc_set_schedule(const fc_schedule* s) {
    if (!s) return FC_EINVAL;
    if (s->gemm_cover < 1 || s->gemm_cover > 64 || s->gemm_split < 0 || s->gemm_split > 16 ||
        s->tc_split < 0 || s->tc_split > 1 || s->tc_min_log2 < 10 || s->tc_min_log2 > 40 ||
        s->workers < 1 || s->workers > kMaxWorkers || s->order < 0 || s->order > 1)
        return FC_EINVAL;
    g_sched.gemm_cover.store(s->gemm_cover);
    g_sched.gemm_split.store(s->gemm_split);
    g_sched.tc_split.store(s->tc_split);
    g_sched.tc_min_log2.store(s->tc_min_log2);
    g_sched.workers.store(s->workers);
    g_sched.order.store(s->order);
    return FC_OK;
}

int fc_solve_batched(int count, const fc_handle* h, const fc_cp* rhs, fc_cp* u,
                     const fc_solve_opts* opts, fc_solve_info* info, void* stream) {
    if (count < 0 || (count > 0 && (!h || !rhs || !u || !info))) return FC_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!h[i]) return FC_EINVAL;
        for (int j = 0; j < i; ++j)
            if (h[j] == h[i]) return FC_EINVAL;   // a handle's workspace serves one solve at a time
    }
    if (count == 0) return FC_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FC_ECUDA;
    const int nworkers = std::min(count, std::max(1, sched(g_sched.workers)));
    cudaStream_t ws[kMaxWorkers];
    if (int rc = worker_streams(dev, nworkers, ws)) return rc;
    // the order the workers take the problems in: as given, or (schedule field order) the
    // largest first, n^d then right-hand-side rank, so that no large solve starts last
    std::vector<int> seq(count);
    for (int i = 0; i < count; ++i) seq[i] = i;
    if (sched(g_sched.order) == 1) {
        auto size = [&](int i) { return std::pow((double)h[i]->n, h[i]->d); };
        std::stable_sort(seq.begin(), seq.end(), [&](int a, int b) {
            if (size(a) != size(b)) return size(a) > size(b);
            return rhs[a].rank > rhs[b].rank;
        });
    }
    // fork: every worker stream starts after the work already queued on the caller's stream
    cudaStream_t caller = (cudaStream_t)stream;
    cudaEvent_t fork;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CK(cudaEventRecord(fork, caller));
    for (int i = 0; i < nworkers; ++i) CK(cudaStreamWaitEvent(ws[i], fork, 0));
    std::vector<int> rc(count, FC_OK);
    // a bounded pool of host threads takes the problems in order (each solve is a chain of
    // small launches and stream synchronisations: one host thread per solve in flight)
    std::atomic<int> next{0};
    std::vector<std::thread> workers;
    workers.reserve(nworkers);
    for (int w_ = 0; w_ < nworkers; ++w_)
        workers.emplace_back([&, w_]() {
            if (cudaSetDevice(dev) != cudaSuccess) {
                for (int q; (q = next.fetch_add(1)) < count;) rc[seq[q]] = FC_ECUDA;
                return;
            }
            for (int q; (q = next.fetch_add(1)) < count;) {
                const int i = seq[q];
                std::memset(&info[i], 0, sizeof(fc_solve_info));
                rc[i] = fc_solve(h[i], &rhs[i], &u[i], opts ? &opts[i] : nullptr, &info[i], ws[w_]);
                if (rc[i] != FC_OK && info[i].status == FC_OK) info[i].status = rc[i];
            }
        });
    for (auto& t : workers) t.join();
    // join: the caller's stream waits for every worker stream
    int out = FC_OK;
    for (int i = 0; i < nworkers && out == FC_OK; ++i) {
        cudaEvent_t done;
        cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(done, ws[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, done, 0);
        cudaEventDestroy(done);
        if (e != cudaSuccess) out = cuda_fail(e);
    }
    cudaEventDestroy(fork);
    if (out != FC_OK) return out;
    for (int i = 0; i < count; ++i)
        if (rc[i] != FC_OK) return rc[i];
    return FC_OK;
}

int fc_to_full(fc_handle h, const fc_cp* x, double* dev_dense, void* stream) {
    if (!h || !dev_dense || !check_cp(h, x, false)) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    launch_to_full(st, h->d, h->n, x->rank, x->xi, x->U[0], x->U[1], h->d == 3 ? x->U[2] : x->U[1],
                   x->ld, dev_dense);
    CKL();
    CK(cudaStreamSynchronize(st));
    return FC_OK;
}

int fc_full_solve(fc_handle h, const double* dev_rhs, double* dev_u, double* dev_tmp, void* stream) {
    if (!h || !dev_rhs || !dev_u || !dev_tmp) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = h->n;
    if (h->twid && !h->V) {
        // fast sine transforms: forward passes over axes 0 .. d-2, then the last axis forward,
        // divided by g and back in one pass, then the inverse passes (F = F^-1)
        const SymbolSpec& g = h->spec;
        const int d = h->d;
        launch_dst_pass(st, dev_rhs, dev_u, d, 0, n, h->twid, false, h->lam, n, 0, 0, 0, 0, 0);
        if (d == 2) {
            launch_dst_pass(st, dev_u, dev_u, d, 1, n, h->twid, true, h->lam, n, g.a, g.sn, g.b,
                            g.sp, g.c);
        } else {
            launch_dst_pass(st, dev_u, dev_u, d, 1, n, h->twid, false, h->lam, n, 0, 0, 0, 0, 0);
            launch_dst_pass(st, dev_u, dev_u, d, 2, n, h->twid, true, h->lam, n, g.a, g.sn, g.b,
                            g.sp, g.c);
            launch_dst_pass(st, dev_u, dev_u, d, 1, n, h->twid, false, h->lam, n, 0, 0, 0, 0, 0);
        }
        launch_dst_pass(st, dev_u, dev_u, d, 0, n, h->twid, false, h->lam, n, 0, 0, 0, 0, 0);
        CKL();
        CK(cudaStreamSynchronize(st));
        return FC_OK;
    }
    LdSine F{h->sintab, 2 * (n + 1)};
    const long long nn = (long long)n * n;
    // y = (T_1 x .. x T_d) x  by d axis passes: T_l the DST-I (symmetric), or for per-mode
    // eigenbases V_l^T (forward) and V_l (back)
    auto dst_all = [&](const double* in, double* out, bool forward) -> int {
        if (!h->V) {
            if (h->d == 2) {
                gemm(st, n, n, n, F, LdN{in, n, 0}, 1.0, 0.0, dev_tmp, n);            // axis 0
                gemm(st, n, n, n, LdN{dev_tmp, n, 0}, F, 1.0, 0.0, out, n);           // axis 1
            } else {
                gemm(st, n, (int)nn, n, F, LdN{in, n, 0}, 1.0, 0.0, dev_tmp, n);      // axis 0
                gemm(st, n, n, n, LdN{dev_tmp, n, nn}, F, 1.0, 0.0, out, n, nn, n);   // axis 1 per i3
                gemm(st, (int)nn, n, n, LdN{out, (int)nn, 0}, F, 1.0, 0.0, dev_tmp, (int)nn);  // axis 2
                CK(cudaMemcpyAsync(out, dev_tmp, sizeof(double) * nn * n, cudaMemcpyDeviceToDevice, st));
            }
            return FC_OK;
        }
        const double* V0 = h->V;
        const double* V1 = h->V + nn;
        const double* V2 = h->V + 2 * nn;
        const long long cols0 = (h->d == 2) ? n : nn;
        // axis 0: T_0 x ;  axes 1, 2: x T^T, i.e. x V (forward) or x V^T (back)
        if (forward) gemm(st, n, (int)cols0, n, LdT{V0, n, 0}, LdN{in, n, 0}, 1.0, 0.0, dev_tmp, n);
        else gemm(st, n, (int)cols0, n, LdN{V0, n, 0}, LdN{in, n, 0}, 1.0, 0.0, dev_tmp, n);
        const int b1 = (h->d == 2) ? 1 : n;
        if (forward) gemm(st, n, n, n, LdN{dev_tmp, n, nn}, LdN{V1, n, 0}, 1.0, 0.0, out, n, nn, b1);
        else gemm(st, n, n, n, LdN{dev_tmp, n, nn}, LdT{V1, n, 0}, 1.0, 0.0, out, n, nn, b1);
        if (h->d == 3) {
            if (forward) gemm(st, (int)nn, n, n, LdN{out, (int)nn, 0}, LdN{V2, n, 0}, 1.0, 0.0, dev_tmp, (int)nn);
            else gemm(st, (int)nn, n, n, LdN{out, (int)nn, 0}, LdT{V2, n, 0}, 1.0, 0.0, dev_tmp, (int)nn);
            CK(cudaMemcpyAsync(out, dev_tmp, sizeof(double) * nn * n, cudaMemcpyDeviceToDevice, st));
        }
        return FC_OK;
    };
    int rc = dst_all(dev_rhs, dev_u, true);
    if (rc) return rc;
    launch_full_scale(st, h->d, n, h->lam, n, h->spec.a, h->spec.sn, h->spec.b, h->spec.sp,
                      h->spec.c, dev_u);
    rc = dst_all(dev_u, dev_u, false);
    if (rc) return rc;
    CKL();
    CK(cudaStreamSynchronize(st));
    return FC_OK;
}

void fc_destroy(fc_handle h) {
    if (!h) return;
    if (h->tables) cudaFree(h->tables);
    if (h->ctab) cudaFree(h->ctab);
    if (h->hbuf) cudaFreeHost(h->hbuf);
    if (h->hint) cudaFreeHost(h->hint);
    delete h;
}

}  // extern "C"
