// Measurement helper (not part of the method): the device's sustained FP64
// fused multiply-add rate, the ceiling of kernels bound by GB300's FP64 pipe
// (the batched solver, whose tableaux never leave shared memory).
//
// Every thread runs kChains independent dependency chains of fma(a, x, y); x
// and y come from kernel arguments, so nothing folds at compile time, and each
// chain's result is stored, so nothing is dead.  The rate is
// blocks x threads x kChains x iters / (CUDA-event time of the launch).
#include <cuda_runtime.h>

#include "tabsimplex.h"
#include "tsx_host.h"

namespace {

constexpr int kChains = 8;

__global__ void k_fma_chains(double* out, long long iters, double x, double y) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (long long t = 0; t < iters; ++t) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same chains with only `lanes` lanes of each warp active (op 0: fma,
// op 1: IEEE division): how the pipe charges partial warps and divisions.
__global__ void k_op_chains(double* out, long long iters, double x, double y, int lanes, int op) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + (double)(threadIdx.x + k) * 1e-3;
    if ((int)(threadIdx.x & 31) < lanes) {
        if (op == 0) {
            for (long long t = 0; t < iters; ++t) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], x, y);
            }
        } else {
            for (long long t = 0; t < iters; ++t) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __ddiv_rn(y, a[k]);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" lp_status lp_measure_fp64_op_rate(int op, int lanes, int blocks, int threads, long long iters,
                                             void* stream, double* ms_out, double* warp_ops_per_s_out) {
    if ((op != 0 && op != 1) || lanes < 1 || lanes > 32 || blocks <= 0 || threads <= 0 || threads > 1024 ||
        threads % 32 || iters <= 0) {
        tsx::set_error("lp_measure_fp64_op_rate: need op 0 or 1, lanes 1..32, blocks > 0, threads a multiple "
                       "of 32 up to 1024, iters > 0");
        return LP_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* out = nullptr;
    TSX_CUDA_TRY(cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads), LP_ERR_NOMEM);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lp_status rc = LP_OPTIMAL;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        tsx::set_error("lp_measure_fp64_op_rate: cudaEventCreate failed");
        rc = LP_ERR_CUDA;
    } else {
        cudaEventRecord(e0, s);
        k_op_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999999, op == 0 ? 1e-7 : 3.0, lanes, op);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            tsx::set_error("lp_measure_fp64_op_rate: %s", cudaGetErrorString(e));
            rc = LP_ERR_CUDA;
        } else {
            cudaEventElapsedTime(&ms, e0, e1);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != LP_OPTIMAL) return rc;
    if (ms_out) *ms_out = ms;
    if (warp_ops_per_s_out)
        *warp_ops_per_s_out = (double)blocks * (threads / 32) * kChains * (double)iters / (ms * 1e-3);
    return LP_OPTIMAL;
}

extern "C" lp_status lp_measure_fp64_fma_rate(int blocks, int threads, long long iters, void* stream,
                                              double* ms_out, double* fma_per_s_out) {
    if (blocks <= 0 || threads <= 0 || threads > 1024 || threads % 32 || iters <= 0) {
        tsx::set_error("lp_measure_fp64_fma_rate: need blocks > 0, threads a multiple of 32 up to "
                       "1024, iters > 0");
        return LP_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* out = nullptr;
    TSX_CUDA_TRY(cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads), LP_ERR_NOMEM);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lp_status rc = LP_OPTIMAL;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        tsx::set_error("lp_measure_fp64_fma_rate: cudaEventCreate failed");
        rc = LP_ERR_CUDA;
    } else {
        // x slightly below 1 and y small keep every chain finite and normal
        cudaEventRecord(e0, s);
        k_fma_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            tsx::set_error("lp_measure_fp64_fma_rate: %s", cudaGetErrorString(e));
            rc = LP_ERR_CUDA;
        } else {
            cudaEventElapsedTime(&ms, e0, e1);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != LP_OPTIMAL) return rc;
    if (ms_out) *ms_out = ms;
    if (fma_per_s_out) *fma_per_s_out = (double)blocks * threads * kChains * (double)iters / (ms * 1e-3);
    return LP_OPTIMAL;
}
