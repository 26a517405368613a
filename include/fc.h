/*
 * fc.h — C ABI of libfc, a GB300 (sm_103a) library for the low-rank PCG solve of the
 * fractional optimal-control equation
 *
 *        (beta^2 A^-alpha + gamma A^alpha) u = b,      b = beta * y_Omega,
 *
 * of Heidel, Khoromskaia, Khoromskij and Schulz, "Tensor product method for fast solution
 * of optimal control problems with fractional multidimensional Laplacian in constraints"
 * (arXiv:1809.01971).  Multiplying eqn:forControl (Section 3.1) by beta gives this form.
 *
 * A is the finite-difference Dirichlet Laplacian on the n^d interior grid of (0,1)^d,
 * h = 1/(n+1) (Section 3.2): A = sum_l I x .. x A_(l) x .. x I, A_(l) = h^-2 tridiag(-1,2,-1),
 * A_(l) = F Lambda F with F the orthonormal DST-I, F[j,k] = sqrt(2/(n+1)) sin(pi j k/(n+1)),
 * lambda_k = (4/h^2) sin^2(pi k/(2(n+1))) (eqn:eig_lap).
 *
 * Conventions for every entry point
 *  - All pointers named dev_* or held in fc_cp are DEVICE pointers; *_host are host pointers.
 *    The caller owns every buffer it passes (including the workspace).  The handle owns only
 *    its setup tables, which fc_setup allocates with cudaMalloc and fc_destroy frees.
 *  - A CP (canonical) tensor (eqn:CP_form, Section 5) is
 *        T = sum_{r<rank} xi[r] U_1[:,r] (x) ... (x) U_d[:,r],
 *    with xi (length >= cap) and factor matrices U_l (column-major, leading dimension ld >= n,
 *    at least cap columns) in FP64 device memory.  Columns need not be normalised on input.
 *  - Outputs whose cap is too small get FC_ERANK and y->rank set to the rank needed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *    enqueued on it; entry points that return a value to the host (fc_inner, fc_truncate's
 *    rank, fc_solve) synchronise that stream before returning.  Outputs are undefined on error.
 *  - Return value: FC_OK (0) or a negative FC_E* code; fc_strerror() names it.  No C++
 *    exception crosses the ABI, no kernel traps; CUDA errors are mapped to FC_ECUDA.
 */
#ifndef FC_H
#define FC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FC_OK = 0,
    FC_EINVAL = -1,       /* bad argument (d, n, alpha, beta, gamma, eps, null pointer)   */
    FC_ERANK = -2,        /* output capacity too small / rank cap overflow                */
    FC_ENOCONV = -3,      /* PCG reached k_max before the tolerance                       */
    FC_EBREAKDOWN = -4,   /* <P,S> <= 0: truncation destroyed positive definiteness       */
    FC_ENAN = -5,         /* non-finite scalar in the recurrences                          */
    FC_ECUDA = -6,        /* CUDA runtime error (message via fc_last_cuda_error)           */
    FC_EWORKSPACE = -7,   /* no workspace bound, or bound workspace too small              */
    FC_ESETUP = -8,       /* quadrature / preconditioner construction failed               */
    FC_ETIMEOUT = -9      /* a bounded wait inside a kernel expired (the kernel freed its  */
                          /* resources and returned; results of the call are undefined)     */
};

typedef struct fc_ctx* fc_handle;

/* CP tensor descriptor (eqn:CP_form).  d in {2,3}; all modes have the same size n. */
typedef struct fc_cp {
    int d;
    int n;
    int rank;      /* number of terms (input: used; output: written)            */
    int cap;       /* allocated number of columns / weights                      */
    int ld;        /* leading dimension of every U[l], ld >= n                   */
    double* xi;    /* device, cap weights                                        */
    double* U[3];  /* device, U[l] is ld x cap column-major; U[2] unused if d==2 */
} fc_cp;

/* Setup options; pass NULL for defaults (values in brackets). */
typedef struct fc_setup_opts {
    double delta_sym;   /* target relative accuracy of the operator symbol [1e-10]          */
    int precond_rank;   /* rank R_P of the exponential-sum preconditioner fit [24]           */
    int max_rank;       /* largest CP rank of any iterate after truncation [32]              */
    int max_tucker;     /* largest Tucker rank per mode inside the truncation [48]           */
    int max_input_rank; /* largest rank of a right-hand side / fc_apply input [max_rank]     */
    int directional;    /* != 0: the directionally fractional operator A_(alpha) =           */
                        /* sum_l (-Delta_l)^alpha (Remark after Lemma 4.1) in place of A^alpha: */
                        /* the equation (beta^2 A_(alpha)^-1 + gamma A_(alpha)) u = b [0]    */
    int precision;      /* 0: FP64 contractions; 1: the large contractions (DST, Khatri-Rao  */
                        /* projections, Tucker core) in double-float arithmetic on the FP32  */
                        /* pipe (hi + lo FP32 pairs, ~1e-14 relative), 64x GB300's FP64 rate; */
                        /* 2: contractions of >= 2^tc_min_log2 (fc_schedule) multiply-adds on */
                        /* the BF16 tensor cores                                              */
                        /* as exact products of 7-bit fixed-point digits of the FP64 operands */
                        /* (8 digits, FP32-exact accumulation, error below FP64 rounding of  */
                        /* the row/column scales), the truncation's Grams and bases and the  */
                        /* inner products' cross-Grams included.  The small eigen-solves and  */
                        /* Cholesky factors and the PCG scalars stay FP64 in every form, and  */
                        /* form 1 keeps the Grams of the truncation FP64 [0]                  */
    int op_kind;        /* operator (Section 6, Tables 6.1-6.4): 0 the control operator      */
                        /* beta^2 A^-alpha + gamma A^alpha (A^alpha + A^-alpha at beta =      */
                        /* gamma = 1); 1 A^alpha; 2 I + A^(2 alpha) (needs 2 alpha <= 1).     */
                        /* beta, gamma enter only kind 0; fc_state needs kind 0 [0]           */
    int precond_kind;   /* 0: least-squares exponential sum of 1/g (rank precond_rank);       */
                        /* 1: the sinc-quadrature sum of rho^-alpha (the symbol g_1 of        */
                        /* Section 6, the exact inverse of A^alpha) [0]                        */
    const double* coeff[3]; /* host, per mode NULL (constant 1) or n+1 values a_l((i+1/2) h),   */
                        /* i = 0..n, all > 0: the mode-l operator is the stiffness matrix of   */
                        /* -(a_l u')' (Remark on variable coefficients), whose orthonormal     */
                        /* eigenvectors (implicit-QR tridiagonal eigen-solve at setup, O(n^3)) */
                        /* replace the DST-I of that mode and whose eigenvalues the spectrum   */
                        /* [NULL]                                                              */
} fc_setup_opts;

typedef struct fc_setup_info {
    int n, d;
    int rank_symbol;    /* R_A = R_minus + d * R_plus (eqn:Func_of_rho, Lemma 4.1)           */
    int rank_minus;     /* nodes of the exponential sum for rho^-alpha                        */
    int rank_plus;      /* nodes of the exponential sum for rho^(alpha-1)                     */
    int rank_precond;   /* R_P                                                                */
    double rho_min, rho_max;
    double sym_err;     /* max relative error of the symbol on a geometric rho grid          */
    double pc_err;      /* max |p(rho) g(rho) - 1| of the preconditioner on that grid        */
    size_t workspace_bytes;
} fc_setup_info;

typedef struct fc_solve_opts {
    double tol;         /* stop when ||R||/||B|| <= tol (recursive residual) [1e-8]          */
    double eps;         /* truncation accuracy; <= 0 means the eps given to fc_setup         */
    int kmax;           /* iteration limit [100]                                              */
    int max_rank;       /* CP rank cap of the iterates; <= 0 means the fc_setup value         */
    int spectral;       /* != 0: spectral-resident iteration: B is transformed once (DST-I of  */
                        /* its factors), every iterate stays in the eigenbasis where symbol    */
                        /* and preconditioner are diagonal and inner products are unchanged    */
                        /* (F orthogonal), and X is transformed back once at exit; the same    */
                        /* result without the two DSTs per mat-vec [0]                          */
    int precision;      /* contraction form of this solve: 0 the handle's (fc_setup_opts.      */
                        /* precision); 1 FP64, 2 double-float FP32, 3 tensor-core digits, so   */
                        /* one set-up serves every form [0]                                     */
    int stall;          /* > 0: stop with FC_ENOCONV once `stall` iterations in a row have not */
                        /* brought ||R||/||B|| 10% below the last value that did (truncated    */
                        /* iterates reach a floor set by eps and the rank caps), and return    */
                        /* the iterate with the smallest recursive residual (also at kmax);    */
                        /* 0: Algorithm 1 as stated, stop at tol or kmax only [0]              */
} fc_solve_opts;

typedef struct fc_solve_info {
    int status;         /* FC_OK, FC_ENOCONV, FC_EBREAKDOWN, FC_ENAN                          */
    int iters;
    double relres;      /* last recursive ||R^(k+1)|| / ||B|| (with stall detection on an     */
                        /* unconverged exit: that of the returned iterate)                      */
    int rank_x;         /* CP rank of the returned solution                                   */
    int max_rank_seen;  /* largest CP rank of any truncated iterate                           */
    int trunc_calls;
    int tucker_max;     /* largest Tucker rank r_l chosen by any truncation of the solve      */
    double tucker_mean; /* mean Tucker rank over all truncations and modes                    */
    int basis_max;      /* largest orthonormal sketch basis (live columns) of any truncation */
    double history[128];/* relres per iteration (first min(iters,128))                       */
} fc_solve_info;

/* Build the spectrum (eqn:eig_lap), the CP symbol of beta^2 rho^-alpha + gamma rho^alpha by
 * sinc quadrature of the Laplace transform (Section 4.2, eqn:Sinc_quadr_trunc, eqn:Func_of_rho;
 * the positive power through Lemma 4.1), and the exponential-sum preconditioner of 1/g.
 * Requires 0 < alpha <= 1, beta > 0, gamma > 0, d in {2,3}, 1 <= n <= 8191, eps > 0.
 * Allocates the handle's device tables (cudaMalloc on the current device). */
int fc_setup(int n, int d, double alpha, double beta, double gamma, double eps,
             const fc_setup_opts* opts, fc_handle* out);

/* Sizes and accuracy figures of a handle. */
int fc_get_info(fc_handle h, fc_setup_info* info);

/* Bytes of device scratch that fc_apply/fc_precond/fc_truncate/fc_inner/fc_solve need. */
int fc_workspace_size(fc_handle h, size_t* bytes);

/* Bind caller-owned device scratch (>= fc_workspace_size bytes, 256-byte aligned). The
 * handle keeps the pointer; calls on one handle must not overlap in time. */
int fc_set_workspace(fc_handle h, void* dev_ptr, size_t bytes);

/* Copy the operator symbol (which=0), the preconditioner symbol (which=1) or the state symbol
 * beta rho^-alpha (which=2, eqn:State) as a CP tensor
 * in the eigen-index domain: diag(g(Lambda)) ~ sum_k xi_k E_1[:,k] x .. x E_d[:,k] with
 * E_l[i,k] a function of lambda_i (eqn:Func_of_rho).  out->cap must be >= the symbol rank. */
int fc_get_symbol(fc_handle h, int which, fc_cp* out, void* stream);

/* y = (beta^2 A^-alpha + gamma A^alpha) x in CP form, untruncated: rank R_A * x->rank,
 * term (k, j) at column k * x->rank + j (eqn:Lap2DtimesX / eqn:Lap3DtimesX, Section 3.2):
 * y = sum_{k,j} xi_k eta_j (x)_l F (e_lk . F x_lj).  The DST runs as a sine-matrix product. */
int fc_apply(fc_handle h, const fc_cp* x, fc_cp* y, void* stream);

/* y = P(A) x with the rank-R_P preconditioner symbol (Section 3.3, precond of Algorithm 1);
 * rank R_P * x->rank, same layout as fc_apply. */
int fc_precond(fc_handle h, const fc_cp* x, fc_cp* y, void* stream);

/* y = trunc(x, eps) (Section 5: RHOSVD canonical -> Tucker -> canonical; d=2 the reduced
 * SVD).  Per mode the leading left singular subspace of the weighted side matrix
 * U_l diag(|xi|) is kept up to eps ||xi||_2 / sqrt(2d) in Frobenius norm (at most max_tucker
 * columns), the Tucker core is formed, and its canonical terms (d=3: mode-3 rotation then
 * slice SVDs) are dropped smallest first while their norm stays <= eps ||core|| / sqrt(2),
 * keeping at most max_rank.  normalize != 0 first rescales every column to unit norm.
 * Result columns are unit vectors, weights positive and descending.  Synchronises. */
int fc_truncate(fc_handle h, const fc_cp* x, double eps, int max_rank, int normalize,
                fc_cp* y, void* stream);

/* y = trunc(F(A) x, eps) as one fused step (the lines S = trunc(fun(P)) and
 * Z = trunc(precond(R)) of Algorithm 1): which = 0 applies the operator symbol, which = 1 the
 * preconditioner, which = 2 the state operator beta A^-alpha (see fc_state).  The R_A * x->rank (or R_P * x->rank) Khatri-Rao columns of the mat-vec are
 * never formed in HBM: the truncation (same rule as fc_truncate with normalize = 0) reads them
 * implicitly in the eigen-index domain and applies the inverse DST-I only to the r_l Tucker
 * basis columns (F is orthogonal, Section 3.2).  x->rank <= max_input_rank.  Synchronises. */
int fc_apply_trunc(fc_handle h, int which, const fc_cp* x, double eps, int max_rank, fc_cp* y,
                   void* stream);

/* State recovery (eqn:State, eqn:L_alp_state): y = trunc(beta A^-alpha u, eps), with the
 * beta^2 rho^-alpha part of the operator symbol divided by beta (R_minus terms); same layout
 * and truncation rule as fc_apply_trunc.  (The adjoint of the KKT system is p = (gamma/beta) u:
 * u with its weights scaled.)  For a handle set up with `directional`, A_(alpha)^-1. */
int fc_state(fc_handle h, const fc_cp* u, double eps, int max_rank, fc_cp* y, void* stream);

/* *out_host = <x, y> = sum_{k,j} xi_k eta_j prod_l <x_lk, y_lj> (inner products of
 * Algorithm 1).  Synchronises. */
int fc_inner(fc_handle h, const fc_cp* x, const fc_cp* y, double* out_host, void* stream);

/* Algorithm 1 (low-rank PCG, Section 3.3) with X^(0) = 0 for L u = rhs, L the handle's operator
 * (beta^2 A^-alpha + gamma A^alpha unless fc_setup_opts.op_kind selects a test operator);
 * every update is truncated with fc_truncate's rule.  u->cap >= max_rank.
 * Returns FC_OK or the failure status (also in info->status). */
int fc_solve(fc_handle h, const fc_cp* rhs, fc_cp* u, const fc_solve_opts* opts,
             fc_solve_info* info, void* stream);

/* `count` independent solves (each as fc_solve on its own handle, right-hand side rhs[i],
 * solution u[i], options opts[i] (opts may be NULL), info[i]), run concurrently.  A pool of
 * host threads (fc_schedule.workers, 16 unless set or tuned) takes the problems in the given
 * order or largest first (fc_schedule.order); each thread drives Algorithm 1 on a non-blocking
 * worker stream of the library's own (per device, created on first use, kept until exit).  The worker streams start after the work already queued on `stream`, and
 * `stream` waits for them before later work on it runs; the call returns when every solve has
 * finished.  A single solve keeps only a few of the 152 SMs busy (its small eigen-solves run
 * on one CTA each), so independent problems overlap on the device.  Handles must be pairwise
 * distinct (FC_EINVAL otherwise: a handle's workspace serves one solve at a time); the calling
 * thread's current device is used.  Returns FC_OK if every solve returned FC_OK, else the
 * first failing problem's code; info[i].status holds each problem's own status.  The worker
 * streams overlap only if they get hardware work queues of their own: CUDA gives 8 unless
 * CUDA_DEVICE_MAX_CONNECTIONS is set (up to 32) before the context is created. */
int fc_solve_batched(int count, const fc_handle* h, const fc_cp* rhs, fc_cp* u,
                     const fc_solve_opts* opts, fc_solve_info* info, void* stream);

/* Launch schedule of the contraction kernels and of fc_solve_batched, process-wide.  The
 * paper has no counterpart: these are the tile shapes, K splits and batch policy that the
 * autotuner below chooses by measurement.  Every schedule gives the same solution up to the
 * rounding order of the contractions' sums.  Defaults in brackets. */
typedef struct fc_schedule {
    int gemm_cover;     /* FP64 / double-float GEMM tile: the largest of 64, 32, 16 whose      */
                        /* launch has at least gemm_cover * 152 / 8 output tiles (double-float: */
                        /* a quarter of that); 1..64 [8]                                        */
    int gemm_split;     /* when those tiles number below 2 * 152, split K (ranges of >= 64)    */
                        /* until about gemm_split CTAs per SM; 0 = never; 0..16 [4]             */
    int tc_split;       /* tensor-core contraction: 1 = K ranges spread over the waves of one   */
                        /* CTA per SM, 0 = fewest K ranges of <= 448; 0..1 [1]                  */
    int tc_min_log2;    /* contraction form 3 sends contractions of >= 2^tc_min_log2           */
                        /* multiply-adds to the tensor cores, smaller ones to the FP64 GEMM;   */
                        /* 10..40 [22]                                                          */
    int workers;        /* fc_solve_batched host threads and worker streams; 1..64 [16]       */
    int order;          /* fc_solve_batched: 0 = problems in the given order, 1 = largest n^d  */
                        /* first (then largest right-hand-side rank); 0..1 [0]                 */
} fc_schedule;

/* Read / replace the process schedule.  fc_set_schedule returns FC_EINVAL (and changes
 * nothing) if a field is out of range; it must not be called while a solve runs in another
 * thread. */
int fc_get_schedule(fc_schedule* out);
int fc_set_schedule(const fc_schedule* s);

/* Cost of one candidate schedule for fc_autotune (lower is better; negative, NaN or infinite:
 * the candidate failed). */
typedef double (*fc_tune_cost)(const fc_schedule* candidate, void* ctx);

/* The autotuner's search, on any cost: coordinate descent from *start (NULL: the process
 * schedule).  Each pass visits the fields in declaration order and evaluates every other value
 * of the field's candidate list with the other fields at their best so far:
 *   gemm_cover {1, 2, 4, 8, 16}, gemm_split {0, 1, 2, 4, 8}, tc_split {0, 1},
 *   tc_min_log2 {20, 22, 24, 26}, workers {8, 16, 24, 32}, order {0, 1};
 * a value is kept when its cost is below (1 - min_gain) times the best cost so far (min_gain in
 * [0, 1): a margin against timing noise).  Stops after `passes` passes (1..8) or after a pass
 * that kept nothing.  The process schedule is not changed.  *best, *best_cost and *evals (cost
 * evaluations, the start's included) may be NULL.  FC_EINVAL: bad arguments, a start out of
 * range, or a start whose cost failed. */
int fc_autotune(const fc_schedule* start, int passes, double min_gain, fc_tune_cost cost,
                void* ctx, fc_schedule* best, double* best_cost, int* evals);

/* The batched form's autotuner: fc_autotune from the process schedule, the cost of a candidate
 * being one fc_solve_batched run of the given problems under it (the candidate is the process
 * schedule during that run): elapsed device time on `stream` (CUDA events around the call) in
 * seconds per converged solve (info status FC_OK); no converged solve is a failed candidate.
 * One untimed run of the start comes first (first-use set-up of streams and kernels).  At exit
 * the process schedule is the best found (also in *best); u holds the last run's solutions.
 * Returns FC_OK, FC_EINVAL (arguments as for fc_solve_batched and fc_autotune), or the first
 * error other than a solve's own status (FC_ENOCONV, FC_EBREAKDOWN, FC_ENAN are costs, not
 * errors); on error the process schedule is restored. */
int fc_autotune_batched(int count, const fc_handle* h, const fc_cp* rhs, fc_cp* u,
                        const fc_solve_opts* opts, int passes, double min_gain,
                        fc_schedule* best, double* best_cost, int* evals, void* stream);

/* Expand a CP tensor to the full n^d array, column-major (i_1 fastest). */
int fc_to_full(fc_handle h, const fc_cp* x, double* dev_dense, void* stream);

/* Full-format eigenbasis solve u = (F x..x F) diag(1/g(rho)) (F x..x F) rhs with the exact
 * symbol of the handle's operator, g(rho) = beta^2 rho^-alpha + gamma rho^alpha for the control
 * operator (eqn:DiagFLaplace3D, Section 3.2);
 * rhs and u are n^d column-major device arrays (may alias). Needs n^d doubles of workspace
 * beyond fc_workspace_size: pass it as dev_tmp. */
int fc_full_solve(fc_handle h, const double* dev_rhs, double* dev_u, double* dev_tmp,
                  void* stream);

/* <x, y> like fc_inner, without a handle and without allocating: for callers that cannot call
 * cudaMalloc (inside a graph capture that must not allocate, hosts that hand out device memory
 * themselves, loops that forbid allocation after start-up).  The paper has no counterpart.
 *  - x, y: CP tensors as in fc_inner (same d and n, d in {2,3}); dev_out: DEVICE pointer that
 *    receives the one double.  Stream-ordered on `stream`; nothing is synchronised.
 *  - Scratch is a file-scope device array of 3 * FC_STATIC_MAX_RANK^2 doubles (384 KiB) that
 *    every GPU which loads the library holds until the process exits; ranks above
 *    FC_STATIC_MAX_RANK return FC_ERANK.  No cudaMalloc, cudaFree or allocating library call.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream capture.  The address
 *    is kept for the life of the process: after cudaDeviceReset on that device, do not call
 *    this entry point again in the same process.
 *  - x, y and dev_out must live on the calling thread's current device.
 *  - All calls share the one array: calls whose work overlaps on the GPU (other streams or
 *    threads) race and must be serialised by the caller. */
#define FC_STATIC_MAX_RANK 128
int fc_inner_static(const fc_cp* x, const fc_cp* y, double* dev_out, void* stream);

void fc_destroy(fc_handle h);
const char* fc_strerror(int code);
const char* fc_last_cuda_error(void);

/* Test hook; the paper has no counterpart.  Sets the iteration limit of the producer-side
 * mbarrier waits of the tensor-core contraction kernel (default 2^24 polls, about 1 s) for the
 * whole process and returns the previous limit in *previous (may be NULL).  With 0 those waits
 * give up at once, so a test sees FC_ETIMEOUT from a tensor-core solve without faulting or
 * hanging the GPU: the kernel stops producing, its MMA-issuing thread still drains the MMAs it
 * issued with the full limit before the tensor memory is freed, and the call returns.
 * iterations < 0: FC_EINVAL. */
int fc_set_wait_limit(int iterations, int* previous);

/* Number of CUDA kernels libfc has launched in this process so far (all handles, all
 * devices); a host-side counter for instrumentation, no synchronisation. */
unsigned long long fc_launch_count(void);

/* Eigen-decomposition of `batch` symmetric m x m FP64 matrices on the device (m <= 64), the
 * small dense eigen-solves of the RHOSVD truncation (Section 5).  Matrix b is column-major at
 * dev_A + b*strideA (leading dimension lda; its symmetric part is used); eigenvalues in
 * descending order go to dev_w + b*strideW, orthonormal eigenvectors to the columns of
 * dev_V + b*strideV (leading dimension ldv).  One CTA per matrix; stream-ordered.
 *  method 0: Householder tridiagonalisation, bisection, inverse iteration, back-transformation
 *            (FP64, eigenvalues accurate to ~u ||A|| in absolute terms);
 *  method 1: the truncation's solver for graded positive semi-definite Grams: Jacobi sweeps in
 *            FP32, eigenvectors made orthonormal (to ~1e-14: Gram and product in double-float,
 *            Cholesky factor and its inverse in FP64) by Cholesky-QR in order of
 *            increasing eigenvalue; eigen-directions accurate relative to the grading, the
 *            eigenvalues FP64 Rayleigh quotients of the returned vectors. */
int fc_symeig(int method, int batch, int m, const double* dev_A, int lda, long long strideA,
              double* dev_w, long long strideW, double* dev_V, int ldv, long long strideV,
              void* stream);

/* C = alpha op(A) op(B) + beta C for column-major FP64 device matrices (op(A) M x K, op(B)
 * K x N; op = transpose if transA / transB), in the given contraction form: 0 the FP64 tiled
 * GEMM, 1 double-float on the FP32 pipe, 2 the BF16 tensor cores with 8 fixed-point digits
 * per operand (any size; the solver routes contractions of at least 2^tc_min_log2
 * multiply-adds there, fc_schedule).  This is the contraction kernel of every form of the solver, exposed for testing
 * and reuse: the paper has no counterpart of it.  All pointers are device pointers owned by
 * the caller; lda >= rows of A as stored, etc.  Asynchronous on `stream`; FC_ETIMEOUT (form
 * 2) only after a synchronisation of the stream inside the call.  Errors: FC_EINVAL. */
int fc_dgemm(int precision, int transA, int transB, int M, int N, int K, double alpha,
             const double* dev_A, int lda, const double* dev_B, int ldb, double beta,
             double* dev_C, int ldc, void* stream);

/* Kernel-class instrumentation.  fc_prof_enable(kclass) synchronises the device, clears the
 * counters and, until fc_prof_read, brackets every launch of that class with a pair of CUDA
 * events on its stream and accumulates the class's algorithmic work on the device.
 * kclass: 0 = off, 1 = the small eigen-solver (work = 9 c^3 flops per c x c matrix),
 * 2 = the tensor-core contraction (work = BF16 MMA flops issued: 36 digit-pair products per
 * multiply-add of the FP64 contraction, tiles padded to 128 x N), 3 = the FP64 tiled GEMM
 * (work = 2 flops per multiply-add of its live tiles).
 * fc_prof_read disables it, synchronises, and returns the launches, the summed event time of
 * those launches in ms, and the work (flops). */
int fc_prof_enable(int kclass);
int fc_prof_read(long long* launches, double* total_ms, double* work);

#ifdef __cplusplus
}
#endif
#endif /* FC_H */
