// Autotuner of the launch schedule (fc_schedule): coordinate descent over the tile, split and
// batch-policy fields, on a caller-given cost or on the measured throughput of batched solves.
// Host code only; the schedule itself lives in api.cu and is read by every launch.
#include "../../include/fc.h"
#include "fc_common.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr int kFields = 6;

int& field(fc_schedule& s, int f) {
    switch (f) {
        case 0: return s.gemm_cover;
        case 1: return s.gemm_split;
        case 2: return s.tc_split;
        case 3: return s.tc_min_log2;
        case 4: return s.workers;
        default: return s.order;
    }
}

// Candidate values of each field, in the order they are tried.
const std::vector<int>& candidates(int f) {
    static const std::vector<int> c[kFields] = {
        {1, 2, 4, 8, 16}, {0, 1, 2, 4, 8}, {0, 1}, {20, 22, 24, 26}, {8, 16, 24, 32}, {0, 1}};
    return c[f];
}

bool in_range(const fc_schedule& s) {
    // fc_set_schedule's ranges, checked without touching the process schedule
    return s.gemm_cover >= 1 && s.gemm_cover <= 64 && s.gemm_split >= 0 && s.gemm_split <= 16 &&
           s.tc_split >= 0 && s.tc_split <= 1 && s.tc_min_log2 >= 10 && s.tc_min_log2 <= 40 &&
           s.workers >= 1 && s.workers <= 64 && s.order >= 0 && s.order <= 1;
}

bool failed(double c) { return !(c >= 0.0) || std::isinf(c); }

// Cost of the batched form: seconds of device time per converged solve.
struct BatchedCtx {
    int count;
    const fc_handle* h;
    const fc_cp* rhs;
    fc_cp* u;
    const fc_solve_opts* opts;
    cudaStream_t st;
    cudaEvent_t e0, e1;
    std::vector<fc_solve_info> info;
    int err;               // first error that is not a solve's own status
};

double batched_cost(const fc_schedule* cand, void* vctx) {
    auto* c = static_cast<BatchedCtx*>(vctx);
    if (c->err != FC_OK) return -1.0;
    if (int rc = fc_set_schedule(cand)) { c->err = rc; return -1.0; }
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess) e = cudaEventRecord(c->e0, c->st);
    if (e != cudaSuccess) { c->err = fc::record_cuda_error(e); return -1.0; }
    fc_solve_batched(c->count, c->h, c->rhs, c->u, c->opts, c->info.data(), c->st);
    e = cudaEventRecord(c->e1, c->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(c->e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->e0, c->e1);
    if (e != cudaSuccess) { c->err = fc::record_cuda_error(e); return -1.0; }
    int ok = 0;
    for (int i = 0; i < c->count; ++i) {
        const int s = c->info[i].status;
        if (s == FC_OK) ++ok;
        else if (s != FC_ENOCONV && s != FC_EBREAKDOWN && s != FC_ENAN) { c->err = s; return -1.0; }
    }
    return ok > 0 ? 1e-3 * ms / ok : -1.0;
}

}  // namespace

extern "C" {

int fc_autotune(const fc_schedule* start, int passes, double min_gain, fc_tune_cost cost,
                void* ctx, fc_schedule* best, double* best_cost, int* evals) {
    if (!cost || passes < 1 || passes > 8 || !(min_gain >= 0.0 && min_gain < 1.0)) return FC_EINVAL;
    fc_schedule cur;
    if (start) cur = *start;
    else fc_get_schedule(&cur);
    if (!in_range(cur)) return FC_EINVAL;
    int n = 1;
    double cbest = cost(&cur, ctx);
    if (failed(cbest)) {
        if (evals) *evals = n;
        return FC_EINVAL;
    }
    for (int p = 0; p < passes; ++p) {
        bool kept = false;
        for (int f = 0; f < kFields; ++f) {
            const int was = field(cur, f);
            int keep = was;
            for (int v : candidates(f)) {
                if (v == was) continue;
                fc_schedule cand = cur;
                field(cand, f) = v;
                const double c = cost(&cand, ctx);
                ++n;
                if (!failed(c) && c < (1.0 - min_gain) * cbest) { cbest = c; keep = v; }
            }
            if (keep != was) { field(cur, f) = keep; kept = true; }
        }
        if (!kept) break;
    }
    if (best) *best = cur;
    if (best_cost) *best_cost = cbest;
    if (evals) *evals = n;
    return FC_OK;
}

int fc_autotune_batched(int count, const fc_handle* h, const fc_cp* rhs, fc_cp* u,
                        const fc_solve_opts* opts, int passes, double min_gain,
                        fc_schedule* best, double* best_cost, int* evals, void* stream) {
    if (count < 1 || !h || !rhs || !u || passes < 1 || passes > 8 ||
        !(min_gain >= 0.0 && min_gain < 1.0))
        return FC_EINVAL;
    fc_schedule start;
    fc_get_schedule(&start);
    BatchedCtx c{count, h, rhs, u, opts, (cudaStream_t)stream, nullptr, nullptr,
                 std::vector<fc_solve_info>(count), FC_OK};
    cudaError_t e = cudaEventCreate(&c.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&c.e1);
    if (e != cudaSuccess) {
        if (c.e0) cudaEventDestroy(c.e0);
        return fc::record_cuda_error(e);
    }
    // untimed first run: worker streams and kernel attributes are set up on first use
    int rc = fc_solve_batched(count, h, rhs, u, opts, c.info.data(), c.st);
    if (rc == FC_EINVAL || rc == FC_ECUDA || rc == FC_ETIMEOUT || rc == FC_ERANK ||
        rc == FC_EWORKSPACE)
        c.err = rc;
    fc_schedule found = start;
    double fcost = -1.0;
    if (c.err == FC_OK) {
        rc = fc_autotune(&start, passes, min_gain, batched_cost, &c, &found, &fcost, evals);
        if (c.err == FC_OK && rc != FC_OK) c.err = rc;
    }
    cudaEventDestroy(c.e0);
    cudaEventDestroy(c.e1);
    if (c.err != FC_OK) {
        fc_set_schedule(&start);
        return c.err;
    }
    fc_set_schedule(&found);
    if (best) *best = found;
    if (best_cost) *best_cost = fcost;
    return FC_OK;
}

}  // extern "C"
