// fc_inner_static: the CP inner product <x, y> for callers that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: code running inside a CUDA-graph capture that
// must not allocate, plug-in or embedded hosts whose device memory is handed out by someone
// else, and real-time loops that forbid allocation after start-up.  fc_inner needs a handle,
// and fc_setup allocates the handle's tables; this entry point needs neither.  Its scratch
// (the d cross-Gram matrices X_l^T Y_l and the split-K accumulators inside them) lives in a
// fixed file-scope device array that every GPU loading the library holds until exit.
#include "../../include/fc.h"
#include "fc_common.cuh"
#include "fc_kernels.h"

#include <mutex>

namespace {

constexpr int kMaxDev = 64;

// d * R_x * R_y doubles of cross-Gram matrices: 3 * 128 * 128 * 8 B = 384 KiB per device.
__device__ __align__(256) double g_inner_scratch[3 * FC_STATIC_MAX_RANK * FC_STATIC_MAX_RANK];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDev] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fc::record_cuda_error(e);
    if (dev < 0 || dev >= kMaxDev) return FC_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_inner_scratch);
        if (e != cudaSuccess) return fc::record_cuda_error(e);
        if (!p) return FC_ECUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FC_OK;
}

bool valid(const fc_cp* x) {
    return x && (x->d == 2 || x->d == 3) && x->n >= 1 && x->ld >= x->n && x->rank >= 0 &&
           x->rank <= x->cap && (x->rank == 0 || (x->xi && x->U[0] && x->U[1] &&
                                                   (x->d == 2 || x->U[2])));
}

}  // namespace

extern "C" int fc_inner_static(const fc_cp* x, const fc_cp* y, double* dev_out, void* stream) {
    if (!dev_out || !valid(x) || !valid(y) || x->d != y->d || x->n != y->n) return FC_EINVAL;
    if (x->rank > FC_STATIC_MAX_RANK || y->rank > FC_STATIC_MAX_RANK) return FC_ERANK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (x->rank == 0 || y->rank == 0) {
        cudaError_t e = cudaMemsetAsync(dev_out, 0, sizeof(double), st);
        return e == cudaSuccess ? FC_OK : fc::record_cuda_error(e);
    }
    double* M = nullptr;
    int rc = scratch_for_current_device(&M);
    if (rc != FC_OK) return rc;
    const int d = x->d, n = x->n, Rx = x->rank, Ry = y->rank;
    const long long mm = (long long)Rx * Ry;
    // M_l = X_l^T Y_l (Rx x Ry, ld Rx).  Every entry is written before it is read: a plain
    // store, or (split-K) a zeroing pre-pass followed by atomic accumulation.
    for (int l = 0; l < d; ++l)
        fc::gemm(st, Rx, Ry, n, fc::LdT{x->U[l], x->ld, 0}, fc::LdN{y->U[l], y->ld, 0}, 1.0, 0.0,
                 M + l * mm, Rx);
    fc::launch_inner_reduce(st, d, Rx, Ry, x->xi, y->xi, M, Rx, mm, dev_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FC_OK : fc::record_cuda_error(e);
}
